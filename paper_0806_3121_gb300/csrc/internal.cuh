// Internal declarations shared by the CUDA translation units of libabft.
// Not part of the ABI; see include/abft.h for the public contract.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/abft.h"

namespace abft {

// Capacities of the verify scratch lists (per call).
constexpr int kCapFlags = 4096;    // flagged lines per side
constexpr int kCapCands = 2048;    // candidates merged in shared memory
constexpr int kCapReport = 16384;  // device report entries
constexpr int kMaxErased = 16;     // erased blocks per verify call
constexpr int kMaxInject = 256;    // armed epilogue fault injections

// Counter slots in the scratch region.
enum Counter : int {
  kCntColFlags = 0,
  kCntRowFlags = 1,
  kCntReport = 2,
  kCntOverflow = 3,
  kCntRecoverFlagged = 4,
  kCntCands = 5,
  kNumCounters = 16
};

struct FlagEntry {  // one flagged line
  int32_t a, b;     // column line: (I, j); row line: (i, J)
  int32_t nonfin, pad;
  double re, rw;
};

struct CandEntry {
  int32_t row, col, kind, side;
  double re, rw;
};

struct Erased {
  int32_t n;
  int32_t bi[kMaxErased], bj[kMaxErased];
};

// Everything the device code needs to know about one problem.
struct Plan {
  abft_desc d;
  int64_t nvr, nvc;  // verify blocks along rows / columns
  int64_t R, Cc;     // checksum rows of A / checksum columns of B
  int64_t bs, bc;    // erasure block rows / columns (0 when no grid)
  int er, ec;        // ceil(log2(vb_rows)), ceil(log2(vb_cols))
  double s;          // safety factor
  double f1_col, f2_col, f1_row, f2_row;  // threshold factors
  // Fused observed checksums (tensor-core dtypes): the product's epilogue
  // writes per-tile column partial sums (one per 128 rows) and per-row partial
  // sums over column groups of g = min(vb_cols, 256) columns.
  int fused;
  int64_t g, ngrp, ntr_obs;
  abft_ws_layout L;
};

struct InjectEntry {  // one armed bit flip of an accumulator output
  int32_t row, col, bit, pad;
};
// Header of the injection region: {kInjectMagic, count, 0, 0}, entries follow
// at +16 bytes.  The magic keeps a fresh (uninitialised) workspace disarmed.
constexpr int32_t kInjectMagic = 0x0ABF7C0D;

// Scratch region view.
struct Scratch {
  int32_t* cnt;
  FlagEntry* colf;
  FlagEntry* rowf;
  CandEntry* cand;
  abft_fault* report;
  double* part;  // partial reductions of encode
  size_t part_elems;
};

Scratch scratch_view(const Plan& P, void* ws);
size_t scratch_bytes(const Plan& P);

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Host-side count of kernel launches (abft_kernel_launches()).
void count_launches(int64_t n);

// Launchers (return cudaGetLastError() of the launches).
cudaError_t launch_encode_f64(const Plan& P, const double* A, const double* B, void* ws,
                              cudaStream_t st);
// Encode with its partial sums in a static device array (no workspace scratch).
cudaError_t launch_encode_f64_noalloc(const Plan& P, const double* A, const double* B, void* ws,
                                      cudaStream_t st);
size_t static_encode_part_bytes();
cudaError_t launch_gemm_f64(const Plan& P, const double* A, const double* B, double* C, void* ws,
                            bool checksums, cudaStream_t st);
// Tensor-core dtypes: encode (checksum pieces, norms) and the product
// followed by the fold of E16/F16 into the binary64 E/F.
cudaError_t launch_encode_lp(const Plan& P, const void* A, const void* B, void* ws,
                             cudaStream_t st);
size_t lp_part_bytes(const Plan& P);
cudaError_t launch_gemm_lp(const Plan& P, const void* A, const void* B, float* C, void* ws,
                           bool checksums, cudaStream_t st);
// Operands of the tensor-core product: bf16 planes [0] (single or hi) and [1]
// (lo), K-major A (ld lda) and N-major B (ld ldb), nseg = 1 (bf16) or 3 (split).
struct TcOperands {
  const void* a[2];
  const void* b[2];
  int64_t lda, ldb;
  int nseg;
};
cudaError_t launch_gemm_bf16(const Plan& P, const TcOperands& op, float* C, void* ws,
                             bool checksums, cudaStream_t st);
cudaError_t tc_timeout_flag(int** dev_ptr);

// ---- grouped products (many independent bf16 problems, one launch per step)
// Verify blocks are fixed to the product tile: 128 rows x 256 columns.
constexpr int kGrpVbR = 128, kGrpVbC = 256;

struct GProb {
  int64_t m, n, k, lda, ldb, ldc;
  const void* A;  // bf16 m x k (lda)
  const void* B;  // bf16 k x n (ldb)
  float* C;       // m x n (ldc)
  void* acs;      // bf16 (4 nvr) x acs_ld: e-hi, e-lo, w-hi, w-lo per verify block
  void* bcs;      // bf16 k x bcs_ld: 4 pieces per verify column block
  int64_t acs_ld, bcs_ld, R16, C16;
  float* E16;     // R16 x n
  float* F16;     // m x C16
  float* obs_col;  // [tile row][2][n]
  float* obs_row;  // [row][nvc][2]
  double* nArow;
  double* nAblk;
  double* nBcol;
  double* nBblk;
  float* rowpart;  // m x ceil(k/256)
  float* colpart;  // ceil(k/128) x n
  double* partA;   // 2 nvr x ceil(k/2048)
  double* partB;   // 2 nvc x ceil(k/128)
  int64_t nvr, nvc;
  double f1c, f1r, f2;  // threshold factors (s applied at use)
  // offsets of this problem in the flattened grids
  int64_t tile_off;    // product tiles
  int64_t encA_off;    // A-side encode CTAs (2048 columns x a verify block)
  int64_t encB_off;    // B-side encode CTAs (2048 columns x 128 rows)
  int64_t rows_off;    // rows (row norms, row lines)
  int64_t cols_off;    // columns (column norms)
  int64_t vbr_off;     // verify row blocks
  int64_t vbc_off;     // verify column blocks
  int64_t cline_off;   // column lines (verify block x column)
  int32_t ntm, ntn, ntr, ntc;
};

struct GMaps {  // tensor maps of one problem (global memory, 64-byte aligned)
  alignas(64) CUtensorMap a;
  alignas(64) CUtensorMap acs;
  alignas(64) CUtensorMap b;
  alignas(64) CUtensorMap bcs;
};

cudaError_t make_bf16_map(CUtensorMap* map, const void* ptr, int64_t rows, int64_t cols,
                          int64_t ld, uint32_t box_cols, uint32_t box_rows);
cudaError_t launch_gemm_grouped(const GProb* probs, const GMaps* maps, int count,
                                int64_t t_total, bool checksums, const int32_t* inj_hdr,
                                const InjectEntry* inj, cudaStream_t st);
cudaError_t consume_tc_timeout(cudaStream_t st, bool* timed_out);
cudaError_t launch_verify(const Plan& P, void* C, void* ws, const Erased& er, bool reread,
                          cudaStream_t st);
cudaError_t launch_set_inject(const Plan& P, void* ws, const int64_t* rows, const int64_t* cols,
                              const int32_t* bits, int count, cudaStream_t st);
cudaError_t launch_recover(const Plan& P, void* C, void* ws, int bi, int bj, cudaStream_t st);
cudaError_t launch_inject(const Plan& P, void* C, const int64_t* rows, const int64_t* cols,
                          const int32_t* bits, int count, cudaStream_t st);
cudaError_t launch_erase(const Plan& P, void* C, int bi, int bj, cudaStream_t st);

}  // namespace abft
