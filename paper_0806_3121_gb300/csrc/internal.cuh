// Internal declarations shared by the CUDA translation units of libabft.
// Not part of the ABI; see include/abft.h for the public contract.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/abft.h"

namespace abft {

// Capacities of the verify scratch lists (per call).
constexpr int kCapFlags = 4096;    // flagged lines per side
constexpr int kCapCands = 2048;    // candidates merged in shared memory
constexpr int kCapReport = 16384;  // device report entries
constexpr int kMaxErased = 16;     // erased blocks per verify call
constexpr int kMaxBlockChecksums = 4;  // block checksums of an erasure grid (grid_f)

// Coefficient of block row I in block checksum l of a p-block-row grid:
// x_I^l with distinct dyadic nodes x_I = (2I + 1 - p) / 2^e, 2^e > p,
// symmetric about 0 (every f x f minor of this Vandermonde matrix is
// nonsingular; centring the nodes keeps neighbouring blocks' systems ten
// times better conditioned than nodes in (0, 1); l = 0 is the plain sum).
__host__ __device__ inline double block_coef(int l, int I, int p) {
  int e = 0;
  while ((1 << e) <= p) ++e;
  const double x = ldexp((double)(2 * I + 1 - p), -e);
  double c = 1.0;
  for (int t = 0; t < l; ++t) c *= x;
  return c;
}
constexpr int kMaxInject = 256;    // armed epilogue fault injections

// Counter slots in the scratch region.  Slots below kNumCleared are cleared
// by every verify call; the status words after them belong to the workspace
// and describe its last encode / product (they are read, not cleared, by the
// verify and the group report):
//   kCntTimeout     set by a tensor-core product whose bounded waits gave up
//                   (cleared when the next product on this workspace starts);
//   kCntFp8Inexact  set by an FP8 encode that met a value not exact in bf16
//                   (cleared when the next encode on this workspace starts).
enum Counter : int {
  kCntColFlags = 0,
  kCntRowFlags = 1,
  kCntReport = 2,
  kCntOverflow = 3,
  kCntRecoverFlagged = 4,
  kCntCands = 5,
  kNumCleared = 8,
  kCntTimeout = 8,
  kCntFp8Inexact = 9,
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
  int32_t prob, pad;
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
  int f;             // block checksums of the erasure grid (rows f * bs after the verify rows)
  int er, ec;        // ceil(log2(vb_rows)), ceil(log2(vb_cols))
  double s;          // safety factor
  double f1_col, f2_col, f1_row, f2_row;  // threshold factors
  // Fused observed checksums (tensor-core dtypes): the product's epilogue
  // writes per-tile column partial sums (one per 128 rows) and per-row partial
  // sums over column groups of g = min(vb_cols, 128) columns.
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

// Error reporting of the C ABI: sets the thread-local message, returns st.
abft_status fail(abft_status st, const char* fmt, ...);
abft_status cuda_fail(cudaError_t e, const char* where);

// Detection-threshold factors of a dtype for inner dimension k and verify
// blocks vb_r x vb_c:  tau = s ||line|| (f1 ||block|| + f2 ||checksum||).
void threshold_factors(int dtype, int64_t k, int64_t vb_r, int64_t vb_c, double* f1_col,
                       double* f1_row, double* f2);

// Launchers (return cudaGetLastError() of the launches).
cudaError_t launch_encode_f64(const Plan& P, const double* A, const double* B, void* ws,
                              cudaStream_t st);
// Chained encode: the checksum rows of A carried from the earlier product PL
// (its workspace wsL), and/or the checksum columns of B from PR (wsR); the
// other side encoded as usual.  Writes the carried deviation bounds.
cudaError_t launch_encode_f64_chained(const Plan& P, const double* A, const double* B, void* ws,
                                      const Plan* PL, const void* wsL, const Plan* PR,
                                      const void* wsR, cudaStream_t st);
// Deviation bounds of the checksum rows / columns carried out of an earlier
// product (its plan and workspace), into car (2 per verify block).
cudaError_t launch_carry_rows(const Plan& PL, const void* wsL, double* car, cudaStream_t st);
cudaError_t launch_carry_cols(const Plan& PR, const void* wsR, double* car, cudaStream_t st);
// Chained encode of the split dtypes (binary32 operands, bf16 pieces): the
// operand planes are split from A and B as usual; the carried rows / columns
// are split into the checksum planes instead of forming checksums.
cudaError_t launch_encode_lp_chained(const Plan& P, const void* A, const void* B, void* ws,
                                     const Plan* PL, const void* wsL, const Plan* PR,
                                     const void* wsR, cudaStream_t st);
// Encode with its partial sums in a static device array (no workspace scratch).
cudaError_t launch_encode_f64_noalloc(const Plan& P, const double* A, const double* B, void* ws,
                                      cudaStream_t st);
size_t static_encode_part_bytes();
cudaError_t launch_gemm_f64(const Plan& P, const double* A, const double* B, double* C, void* ws,
                            bool checksums, cudaStream_t st);
// Tensor-core dtypes: encode (checksum pieces, norms) and the product
// followed by the fold of E16/F16 into the binary64 E/F.
cudaError_t launch_encode_lp(const Plan& P, const void* A, const void* B, const void* a_scale,
                             const void* b_scale, void* ws, cudaStream_t st);
size_t lp_part_bytes(const Plan& P);
cudaError_t launch_gemm_lp(const Plan& P, const void* A, const void* B, float* C, void* ws,
                           bool checksums, cudaStream_t st);
// Operands of the tensor-core product: up to three bf16 planes of K-major A
// (ld lda) and N-major B (ld ldb).  The K loop runs nseg segments; segment s
// multiplies A plane (seg_a >> 2s) & 3 by B plane (seg_b >> 2s) & 3.
struct TcOperands {
  const void* a[3];
  const void* b[3];
  int64_t lda, ldb;
  int nseg;
  uint32_t seg_a, seg_b;
  // native FP8 data tiles (a8 == nullptr: none): e4m3 codes of A (m x k, lda8
  // bytes) and of B transposed (b8 = B^T, n x k, ldb8 bytes), 16-byte aligned
  // rows, and their binary32 power-of-two block scales (ceil(m/128) x
  // ceil(k/128), ceil(k/128) x ceil(n/128), row-major, device)
  const void* a8;
  const void* b8;
  int64_t lda8, ldb8;
  const float* sA;
  const float* sB;
  uint32_t* f8grp;  // the data tiles' scale-group words (workspace, written first)
};
// status: the word a timeout is recorded in (cleared on `st` before the
// launch).
cudaError_t launch_gemm_bf16(const Plan& P, const TcOperands& op, float* C, void* ws,
                             bool checksums, int* status, cudaStream_t st);
// Scale groups of the data tiles (128 x 256) of an FP8 product: per tile one bit
// per 128-wide k-step, set where the block-scale product of either 128-column
// half changes (out: ceil(m/128) * ceil(n/256) * ceil(ceil(k/128)/32) words).
cudaError_t launch_f8_groups(const float* sA, const float* sB, int64_t m, int64_t n, int64_t k,
                             uint32_t* out, cudaStream_t st);
// Process-wide word that receives the timeout of a checksum-free product run
// without a workspace (nothing reads it: such a call has no report).
cudaError_t tc_timeout_fallback(int** dev_ptr);

// ---- grouped products (many independent bf16 problems, one launch per step)
// Verify blocks: 128 rows (one product tile row) x 256 columns.
constexpr int kGrpVbR = 128, kGrpVbC = 256, kGrpEr = 7, kGrpEc = 8;

struct GProb {  // one problem of a group, in device memory
  int64_t m, n, k, lda, ldb, ldc;
  const void* A;  // bf16 m x k (lda)
  const void* B;  // bf16 k x n (ldb)
  float* C;       // fp32 m x n (ldc)
  void* acs;      // bf16 R16 x acs_ld: per verify block e-hi, e-lo, w-hi, w-lo rows
  void* bcs;      // bf16 k x bcs_ld: per verify column block the same 4 columns
  int64_t acs_ld, bcs_ld, R16, C16;
  float* E16;      // R16 x n: acs B
  float* F16;      // m x C16: A bcs
  float* obs_col;  // [32-row block][2][n]: observed e/w column sums of each 32 rows
  float* obs_row;  // [row][ngrp][2]: observed e/w row sums of each g-column group
  double* nArow;   // m: ||A_i||
  double* nAblk;   // 4 nvr: threshold norms of each verify row block
  double* nBcol;   // n: ||B_:j||
  double* nBblk;   // 4 nvc
  float* nArow32;  // m: ||A_i|| rounded to fp32 (screening)
  float* nBcol32;  // n
  float* tauA;     // 2 nvr: s (f1c ||A_I||_F + f2 ||e^T A_I||), the same with w (fp32)
  float* tauB;     // 2 nvc: s (f1r ||B_J||_F + f2 ||B_J e||), the same with w
  float* rowpart;  // m x ceil(k/256) squared-norm partials
  float* colpart;  // ceil(k/128) x n
  double* partA;   // 2 nvr x ceil(k/256)
  double* partB;   // 2 nvc x ceil(k/128)
  int64_t nvr, nvc, ngrp;
  double f1c, f1r, f2;  // threshold factors (the safety factor applies at use)
  int32_t nhc, nbc;     // checksum halves (64 rows) / boxes (64 columns)
  int32_t bpt, g;       // boxes per tile (tile width 64 bpt), row-sum group width
  int32_t st_ok;        // bit 0/1/2: TMA store map of C / E16 / F16 valid
  int32_t swap_rows;    // 1: the checksum rows are products of their own (swapped
                        // tiles, see kGrpSwapTile), not halves after the data rows
};

// Tile-list entries of a grouped product are int4 {problem, tile row, tile
// column, kind}.  kind kGrpSwapTile: the expected column checksums E16 = acs B
// of 256 columns of B (tile column = 256-column block) computed with the
// operands' roles swapped -- B's columns on the M side (MN-major, two M = 128
// MMAs), the R16 <= 128 checksum rows on the N side (K-major) -- so the MMAs'
// N is R16 rounded up to 16 instead of a whole 128-row tile of mostly empty
// rows.  Used for problems whose data rows fill whole tiles (an even number of
// 64-row halves).
constexpr int kGrpSwapTile = 1;
// kind kGrpF2Tile: a tile whose columns are all checksum columns (F16 = A bcs
// of its 128 rows): its stages hold two k-steps (A 2 x 16 KiB, the checksum box
// 2 x 8 KiB) instead of one, so it takes half as many stages of the ring.
constexpr int kGrpF2Tile = 2;

struct GMaps {  // tensor maps of one problem (64-byte aligned in device memory)
  CUtensorMap a, acs, b, bcs;   // 64-row halves / one 64-column box
  CUtensorMap a128, acs128;     // 128-row boxes (a whole tile's A)
  CUtensorMap bw[3];            // 2, 3, 4 full 64-column boxes of B in one copy (3-D view)
  CUtensorMap bcs4;             // four full checksum boxes in one copy
  CUtensorMap cst, est, fst;    // fp32 store maps of C, E16, F16 (per GProb::st_ok)
};

// The grouped kernels: CTA b of kernel kk works on problem tab[kk][b].x, its
// local unit tab[kk][b].y.
// Row lines per thread of the grouped row check (k_grp_row).
constexpr int kGrpRowLines = 4;

enum GroupKernel : int {
  kGkEncA = 0,   // A column checksums: nvr x ceil(acs_ld/256)
  kGkEncB,       // B row checksums: ceil(n/256) x ceil(k/128)
  kGkLines,      // line norms: ceil(m/256) + ceil(n/256)
  kGkColCheck,   // column lines: nvr x ceil(n/256)
  kGkRowCheck,   // row lines: ceil(m nvc / (256 kGrpRowLines))
  kGkCount
};

struct GroupDev {  // device view of a bound group (every pointer in the workspace)
  const GProb* probs;
  const GMaps* maps;
  int count;
  const int4* tiles_cs;     // product tiles with checksums
  int64_t ntiles_cs;
  const int4* tiles_plain;  // product tiles without checksums
  int64_t ntiles_plain;
  const int2* tab[kGkCount];
  int64_t nctas[kGkCount];
  double s;                 // threshold safety factor
  int32_t* cnt;             // verify counters
  FlagEntry* colf;          // flagged lines (pad = problem)
  FlagEntry* rowf;
  CandEntry* cand;
  abft_fault* report;
  int32_t* inj_hdr;         // armed epilogue injections
  InjectEntry* inj;
};

cudaError_t make_bf16_map(CUtensorMap* map, const void* ptr, int64_t rows, int64_t cols,
                          int64_t ld, uint32_t box_cols, uint32_t box_rows);
// The 3-D view of a row-major rows x cols bf16 matrix as (64 columns, rows,
// full 64-column box) with a box of `depth` 64 x 64 boxes.
cudaError_t make_bf16_map_boxes(CUtensorMap* map, const void* ptr, int64_t rows, int64_t cols,
                                int64_t ld, int depth);
// fp32 TMA store map of a row-major output (box 32 x 32, 128-byte swizzle);
// *ok = false (no map) when the base or the row pitch is not 16-byte aligned.
cudaError_t make_f32_store_map(CUtensorMap* map, const void* ptr, int64_t rows, int64_t cols,
                               int64_t ld, bool* ok);
cudaError_t launch_group_encode(const GroupDev& G, cudaStream_t st);
cudaError_t launch_group_gemm(const GroupDev& G, bool checksums, cudaStream_t st);
cudaError_t launch_group_verify(const GroupDev& G, cudaStream_t st);
cudaError_t prepare_group_kernels();
// Arms `count` epilogue injections (count = 0 disarms) in the region at hdr.
cudaError_t launch_set_inject_raw(int32_t* hdr, const InjectEntry* entries, int count,
                                  cudaStream_t st);
cudaError_t launch_verify(const Plan& P, void* C, void* ws, const Erased& er, bool reread,
                          cudaStream_t st);
cudaError_t launch_set_inject(const Plan& P, void* ws, const int64_t* rows, const int64_t* cols,
                              const int32_t* bits, int count, cudaStream_t st);
// Rebuilds the erased blocks rows[0..t) of block column bj from the first t
// block checksums (t <= f): minv is the inverse of M[l][u] = block_coef(l,
// rows[u], p), row-major t x t, in binary64.
cudaError_t launch_recover(const Plan& P, void* C, void* ws, int bj, const int* rows, int t,
                           const double* minv, cudaStream_t st);
// One rank's share of a block rebuild over GPUs: out (bs x bc binary64) =
// (with_checksum ? S_bj : 0) - sum of the local blocks of block column bj other
// than block row `skip` (-1: none).
cudaError_t launch_block_partial(const Plan& P, const void* C, const void* ws, int skip, int bj,
                                 bool with_checksum, double* out, cudaStream_t st);
// Writes src (bs x bc binary64) into block (bi, bj) of C and re-checks the
// block's column lines (count in cnt[kCntRecoverFlagged]).
cudaError_t launch_block_restore(const Plan& P, void* C, void* ws, int bi, int bj,
                                 const double* src, cudaStream_t st);
cudaError_t launch_inject(const Plan& P, void* C, const int64_t* rows, const int64_t* cols,
                          const int32_t* bits, int count, cudaStream_t st);
cudaError_t launch_erase(const Plan& P, void* C, int bi, int bj, cudaStream_t st);

}  // namespace abft
