// Checksum encoding for the tensor-core dtypes (section 2.1; the encoded
// operands of Eq. (1)) and the fold of the product's checksum pieces.
//
// Checksums of bf16 data are accumulated in fp32 and fed to the tensor cores
// as a bf16 hi + lo pair (hi = bf16(x), lo = bf16(x - hi); the pair carries x
// to a relative 2^-18), so the product of each piece with B (or of A with
// each piece) is a separate fp32 row (column) of the ABFT product; the fold
// kernel adds the two pieces in binary64 into the E / F layout that the
// verify kernels share with the binary64 path.
//
// acs rows per verify block I: 4I e-hi, 4I+1 e-lo, 4I+2 w-hi, 4I+3 w-lo; then
// two rows (hi, lo) per block checksum row.  bcs is row-major k x (4 nvc)
// with the same piece order per verify column block.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <stdlib.h>

#include <type_traits>

#include "internal.cuh"

namespace abft {
namespace {

constexpr int kThreads = 256;
constexpr int kColsPerCta = 8 * kThreads;  // 2048 columns, 8 per thread (16-byte loads)
constexpr int kRowsPerCtaB = 128;          // rows of B per CTA in the row-checksum pass
constexpr int kRowBatch = 8;               // rows whose loads are in flight together (A pass)
constexpr int kRowBatchB = 16;             // the same for the B pass
constexpr int kEncCols = 256;              // columns of one bf16 encode unit (8 per lane)
constexpr int kEncWarps = kThreads / 32;   // warps sharing a unit's rows
// A pass with asynchronous copies: each warp keeps Ring::kBatches batches of
// kRowBatch rows in flight in its shared-memory ring (one slot per lane and
// row: 16 bytes of bf16, 8 bytes of e4m3), so the loads do not wait on
// registers.  Both keep 8 KiB per warp in flight (3 batches of bf16 rows, 4
// of e4m3 rows; with 2 batches of 8-byte e4m3 rows the passes ran at 3.3-3.7
// TB/s, short of the bytes in flight that the memory latency asks for).
template <bool kF8>
struct Ring {
  using Slot = typename std::conditional<kF8, uint2, uint4>::type;
  static constexpr int kBatches = kF8 ? 4 : 3;
  static constexpr int kBytes = kEncWarps * kBatches * kRowBatch * 32 * (int)sizeof(Slot);
};
static_assert(Ring<true>::kBytes == 64 * 1024 && Ring<false>::kBytes == 96 * 1024, "ring sizes");

// 16-byte asynchronous global -> shared copy; bytes < 16 zero-fills the rest
// (0: nothing is read).  Both addresses 16-byte aligned.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
// All but the N most recent committed groups of this thread have landed.
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sums over the 32 lanes of N values at once (N = 8 or 16; a transposing
// butterfly, N - 1 + log2(32 / N) shuffles): on return lane l holds, in v[0],
// the sum over all lanes of their v[l / (32 / N)].
template <int N>
__device__ __forceinline__ void reduce_rows(float (&v)[N], int lane) {
#pragma unroll
  for (int s = 16, h = N / 2; h >= 1; s >>= 1, h >>= 1) {
    const bool upper = (lane & s) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const float send = upper ? v[i] : v[i + h];
      const float keep = upper ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
#pragma unroll
  for (int o = 16 / N; o >= 1; o >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
}

// Tree sum over the block's threads in fp32, valid in thread 0 (binary64
// arithmetic is kept out of per-element work: GB300's FP64 pipe is narrow).
__device__ __forceinline__ float block_sumf(float v, float* sh) {
  v = warp_sumf(v);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  float t = 0.f;
  if (w == 0) {
    t = lane < kThreads / 32 ? sh[lane] : 0.f;
    t = warp_sumf(t);
  }
  return t;
}

__device__ __forceinline__ void split(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

__device__ __forceinline__ float ldf(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// Eight consecutive elements starting at column c of a row as raw bf16 bits
// (zeros past `len`), unpacked later:
// a row batch in flight costs 4 registers per row instead of 8.
__device__ __forceinline__ uint4 load8raw(const __nv_bfloat16* row, int64_t c, int64_t len) {
  if (c + 8 <= len && ((reinterpret_cast<uintptr_t>(row + c) & 15) == 0))
    return *reinterpret_cast<const uint4*>(row + c);
  uint32_t w[4] = {0u, 0u, 0u, 0u};
  const uint16_t* r16 = reinterpret_cast<const uint16_t*>(row);
#pragma unroll
  for (int q = 0; q < 8; ++q)
    if (c + q < len) w[q >> 1] |= (uint32_t)r16[c + q] << (16 * (q & 1));
  return make_uint4(w[0], w[1], w[2], w[3]);
}

__device__ __forceinline__ void unpack8(const uint4& u, float (&v)[8]) {
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float2 f = __bfloat1622float2(h[q]);
    v[2 * q] = f.x;
    v[2 * q + 1] = f.y;
  }
}

__device__ __forceinline__ void store8(__nv_bfloat16* dst, const __nv_bfloat16 (&v)[8]) {
  *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(v);
}

// Column checksums of A per verify block (fp32 sums, hi/lo pieces), per-row
// partial sums of squares (one per 256 columns) and per-CTA partials of the
// squared norms of the two checksum rows.  Unit = 256 columns (chunk cx) x one
// verify block I: lane = 8 consecutive columns, warp w = rows i0 + w + 8 t;
// the eight warps' column sums meet in shared memory (red: [8][256][2]
// floats).  lpA_rows adds one row (its 1-based position t + 1 in the block)
// into the lane's sums; lpA_finish combines the warps and writes the unit's
// checksum pieces and norm partials.
// A lane's 8 consecutive floats to shared memory as two 16-byte stores (dst
// 16-byte aligned).
__device__ __forceinline__ void st_shared8(float* dst, const float (&v)[8]) {
  reinterpret_cast<float4*>(dst)[0] = make_float4(v[0], v[1], v[2], v[3]);
  reinterpret_cast<float4*>(dst)[1] = make_float4(v[4], v[5], v[6], v[7]);
}

__device__ __forceinline__ void lpA_rows(const float (&v)[8], int t, float sc, float (&se)[8],
                                         float (&sw)[8], float& sq) {
  const float w = (float)(t + 1) * sc;
  sq = 0.f;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    se[q] += v[q];
    sw[q] = fmaf(w, v[q], sw[q]);
    sq = fmaf(v[q], v[q], sq);
  }
}

__device__ __forceinline__ void lpA_finish(const float (&se)[8], const float (&sw)[8],
                                           __nv_bfloat16* __restrict__ acs, int64_t ldk,
                                           double* __restrict__ part, int64_t nchr, int64_t cx,
                                           int64_t I, float* red, float* sh) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // red: the warps' e sums [warp][column], then their w sums (16-byte stores of
  // a lane's 8 columns; one word per lane and bank-conflict free when read back)
  float* red_w = red + kEncWarps * kEncCols;
  st_shared8(red + warp * kEncCols + 8 * lane, se);
  st_shared8(red_w + warp * kEncCols + 8 * lane, sw);
  __syncthreads();
  const int c = threadIdx.x;  // column of the chunk
  float te = 0.f, tw = 0.f;
#pragma unroll
  for (int w = 0; w < kEncWarps; ++w) {
    te += red[w * kEncCols + c];
    tw += red_w[w * kEncCols + c];
  }
  const int64_t col = cx * kEncCols + c;
  float q0 = 0.f, q1 = 0.f;
  if (col < ldk) {  // columns k .. ldk-1 hold zeros
    __nv_bfloat16 h, l;
    split(te, h, l);
    acs[(4 * I + 0) * ldk + col] = h;
    acs[(4 * I + 1) * ldk + col] = l;
    split(tw, h, l);
    acs[(4 * I + 2) * ldk + col] = h;
    acs[(4 * I + 3) * ldk + col] = l;
    q0 = te * te;
    q1 = tw * tw;
  }
  const float t0 = block_sumf(q0, sh);
  if (threadIdx.x == 0) part[(2 * I) * nchr + cx] = (double)t0;
  const float t1 = block_sumf(q1, sh);
  if (threadIdx.x == 0) part[(2 * I + 1) * nchr + cx] = (double)t1;
  __syncthreads();  // red is reused by the next unit
}

// One unit with register loads (any alignment): kRowBatch rows of loads in
// flight per warp at a time.
__device__ __forceinline__ void lpA_unit(const __nv_bfloat16* __restrict__ A, int64_t lda,
                                         int64_t m, int64_t k, int vb, int e,
                                         __nv_bfloat16* __restrict__ acs, int64_t ldk,
                                         float* __restrict__ rowpart, int64_t nchr,
                                         double* __restrict__ part, int64_t cx, int64_t I,
                                         float* red, float* sh) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t c0 = cx * kEncCols + 8 * lane;
  const float sc = scalbnf(1.0f, -e);
  const int64_t i0 = I * vb, i1 = min(i0 + (int64_t)vb, m);
  const int nrow = (int)(i1 - i0);
  const __nv_bfloat16* Ab = A + i0 * lda;
  float se[8], sw[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) se[q] = sw[q] = 0.f;
  constexpr int kLanesPerRow = 32 / kRowBatch;
  for (int rb = warp; rb < nrow; rb += kEncWarps * kRowBatch) {
    uint4 raw[kRowBatch];
#pragma unroll
    for (int r = 0; r < kRowBatch; ++r) {
      const int t = rb + kEncWarps * r;
      raw[r] = t < nrow ? load8raw(Ab + (int64_t)t * lda, c0, k) : make_uint4(0u, 0u, 0u, 0u);
    }
    float sq[kRowBatch];
#pragma unroll
    for (int r = 0; r < kRowBatch; ++r) {
      float v[8];
      unpack8(raw[r], v);
      lpA_rows(v, rb + kEncWarps * r, sc, se, sw, sq[r]);
    }
    reduce_rows<kRowBatch>(sq, lane);  // row r's sum of squares in lanes r * kLanesPerRow ..
    const int t = rb + kEncWarps * (lane / kLanesPerRow);
    if (lane % kLanesPerRow == 0 && t < nrow) rowpart[(i0 + t) * nchr + cx] = sq[0];
  }
  lpA_finish(se, sw, acs, ldk, part, nchr, cx, I, red, sh);
}

__global__ void __launch_bounds__(kThreads, 2) k_lpA_cols(const __nv_bfloat16* __restrict__ A,
                                                       int64_t lda, int64_t m, int64_t k, int vb,
                                                       int e, __nv_bfloat16* __restrict__ acs,
                                                       int64_t ldk, float* __restrict__ rowpart,
                                                       int64_t nchr, double* __restrict__ part) {
  __shared__ __align__(16) float red[kEncWarps * kEncCols * 2];
  __shared__ float sh[kThreads / 32];
  const int64_t nvb = cdiv(m, vb);
  for (int64_t I = blockIdx.y; I < nvb; I += gridDim.y)
    lpA_unit(A, lda, m, k, vb, e, acs, ldk, rowpart, nchr, part, blockIdx.x, I, red, sh);
}

// Block checksum rows S^(c)[t] = sum_I c_{c,I} A[I*bs + t] (c < f), fp32 sums
// as hi/lo pieces: row c*bs + t of the block checksums -> rows 2 (c*bs + t),
// 2 (c*bs + t) + 1 of S.
__global__ void __launch_bounds__(kThreads) k_lpA_block(const __nv_bfloat16* __restrict__ A,
                                                        int64_t lda, int64_t k, int p, int64_t bs,
                                                        int f, __nv_bfloat16* __restrict__ S,
                                                        int64_t ldk) {
  const int64_t l = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (l >= k) return;
  for (int64_t ct = blockIdx.y; ct < f * bs; ct += gridDim.y) {
    const int c = (int)(ct / bs);
    const int64_t t = ct - c * bs;
    float s = 0.f;
    for (int I = 0; I < p; ++I) s = fmaf((float)block_coef(c, I, p), ldf(A + (I * bs + t) * lda + l), s);
    __nv_bfloat16 h, lo;
    split(s, h, lo);
    S[(2 * ct) * ldk + l] = h;
    S[(2 * ct + 1) * ldk + l] = lo;
  }
}

// Row checksums of B per verify column block (hi/lo pieces in the row-major
// bcs), per-column partial sums of squares (one per 128 rows) and partials
// of the squared norms of the checksum columns.  Verify blocks of 8, 16, ...,
// 256 columns: the lanes of a block reduce with shuffles.  Unit = 256 columns
// (chunk cx) x 128 rows (chunk ry): lane = 8 consecutive columns, warp w = rows
// l0 + w + 8 t; the warps' column squares and block partials meet in shared
// memory (red: [8][256] floats, redq: [8][32][2] floats) in lpB_finish.
__device__ __forceinline__ void lpB_finish(const float (&cs)[8], float q0, float q1, int64_t n,
                                           int vb, float* __restrict__ colpart,
                                           double* __restrict__ part, int64_t nch, int64_t cx,
                                           int64_t ry, float* red, float* redq) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int seg = vb / 8;
  st_shared8(red + warp * kEncCols + 8 * lane, cs);
  redq[(warp * 32 + lane) * 2 + 0] = q0;
  redq[(warp * 32 + lane) * 2 + 1] = q1;
  __syncthreads();
  const int c = threadIdx.x;
  float t = 0.f;
#pragma unroll
  for (int w = 0; w < kEncWarps; ++w) t += red[w * kEncCols + c];
  if (cx * kEncCols + c < n) colpart[ry * n + cx * kEncCols + c] = t;
  if (c < 32 && (c % seg) == 0 && cx * kEncCols + 8 * c < n) {
    float a0 = 0.f, a1 = 0.f;
    for (int w = 0; w < kEncWarps; ++w) {
      a0 += redq[(w * 32 + c) * 2 + 0];
      a1 += redq[(w * 32 + c) * 2 + 1];
    }
    const int64_t Jc = (cx * kEncCols + 8 * c) / vb;
    part[(2 * Jc) * nch + ry] = (double)a0;
    part[(2 * Jc + 1) * nch + ry] = (double)a1;
  }
  __syncthreads();  // red / redq are reused by the next unit
}

// One row of B in a lane's 8 columns: its (e, w) partial sums (reduced over
// the verify block by the caller) and the column squares.
__device__ __forceinline__ void lpB_row(const float (&v)[8], const float (&wq)[8], float (&cs)[8],
                                        float& se, float& sw) {
  se = 0.f;
  sw = 0.f;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    se += v[q];
    sw = fmaf(wq[q], v[q], sw);
    cs[q] = fmaf(v[q], v[q], cs[q]);
  }
}

// The lanes' (e, w) sums of row l reduced over their verify block (seg lanes)
// and stored as hi/lo pieces by the block's first lane.
__device__ __forceinline__ void lpB_store_shfl(float se, float sw, int seg, bool leader, bool valid,
                                               __nv_bfloat16* __restrict__ dst, float& q0,
                                               float& q1) {
  for (int o = seg >> 1; o > 0; o >>= 1) {
    se += __shfl_xor_sync(0xffffffffu, se, o);
    sw += __shfl_xor_sync(0xffffffffu, sw, o);
  }
  if (leader && valid) {
    __nv_bfloat16 pc[4];
    split(se, pc[0], pc[1]);
    split(sw, pc[2], pc[3]);
    *reinterpret_cast<uint2*>(dst) = *reinterpret_cast<const uint2*>(pc);
    q0 = fmaf(se, se, q0);
    q1 = fmaf(sw, sw, q1);
  }
}

// One unit with register loads (any alignment).
__device__ __forceinline__ void lpB_unit(const __nv_bfloat16* __restrict__ B, int64_t ldb,
                                         int64_t k, int64_t n, int vb, int e,
                                         __nv_bfloat16* __restrict__ bcs, int64_t ldcs,
                                         float* __restrict__ colpart, double* __restrict__ part,
                                         int64_t nch, int64_t cx, int64_t ry, float* red,
                                         float* redq) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t c0 = cx * kEncCols + 8 * lane;
  const int64_t l0 = ry * kRowsPerCtaB, l1 = min(l0 + kRowsPerCtaB, k);
  const int seg = vb / 8;  // lanes per verify block (1 .. 32)
  const bool leader = (lane % seg) == 0 && c0 < n;
  const int64_t J = c0 / vb;
  const float sc = scalbnf(1.0f, -e);
  float wq[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) wq[q] = (float)((int)((c0 + q) % vb) + 1) * sc;
  float cs[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) cs[q] = 0.f;
  float q0 = 0.f, q1 = 0.f;
  const int nrow = (int)(l1 - l0);
  const __nv_bfloat16* Bb = B + l0 * ldb;
  for (int rb = warp; rb < nrow; rb += kEncWarps * kRowBatchB) {
    uint4 raw[kRowBatchB];
#pragma unroll
    for (int r = 0; r < kRowBatchB; ++r) {
      const int t = rb + kEncWarps * r;
      raw[r] = t < nrow ? load8raw(Bb + (int64_t)t * ldb, c0, n) : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int r = 0; r < kRowBatchB; ++r) {
      const int64_t l = l0 + rb + kEncWarps * r;
      float v[8], se, sw;
      unpack8(raw[r], v);
      lpB_row(v, wq, cs, se, sw);
      lpB_store_shfl(se, sw, seg, leader, l < l1, bcs + l * ldcs + 4 * J, q0, q1);
    }
  }
  lpB_finish(cs, q0, q1, n, vb, colpart, part, nch, cx, ry, red, redq);
}

__global__ void __launch_bounds__(kThreads, 2) k_lpB_rows(const __nv_bfloat16* __restrict__ B,
                                                       int64_t ldb, int64_t k, int64_t n, int vb,
                                                       int e, __nv_bfloat16* __restrict__ bcs,
                                                       int64_t ldcs, float* __restrict__ colpart,
                                                       double* __restrict__ part, int64_t nch) {
  __shared__ __align__(16) float red[kEncWarps * kEncCols];
  __shared__ float redq[kEncWarps * 32 * 2];
  for (int64_t ry = blockIdx.y; ry < nch; ry += gridDim.y)
    lpB_unit(B, ldb, k, n, vb, e, bcs, ldcs, colpart, part, nch, blockIdx.x, ry, red, redq);
}

// ---------------- streaming encode (16-byte aligned operands and row pitch)
// Persistent CTAs; each warp copies its rows of the CTA's units into its own
// shared-memory ring (one Ring slot per lane and row) with asynchronous copies,
// Ring::kBatches batches of kRowBatch rows ahead of the arithmetic.  The ring
// runs across units, so the loads of the next unit overlap the finishing of
// the current one, and no register holds a load in flight.

struct EncAUnit {  // 256 columns (chunk cx) x verify block I of A
  const __nv_bfloat16* A;
  int64_t lda, m, k;
  int vb, e;
  __nv_bfloat16* acs;
  int64_t ldk;
  float* rowpart;
  int64_t nchr;
  double* part;
  int64_t cx, I;
};
struct EncBUnit {  // 256 columns (chunk cx) x 128 rows (chunk ry) of B
  const __nv_bfloat16* B;
  int64_t ldb, k, n;
  int vb, e;
  __nv_bfloat16* bcs;
  int64_t ldcs;
  float* colpart;
  double* part;
  int64_t nch, cx, ry;
};
// The rows of a unit as the copies see them.
struct RowSrc {
  const __nv_bfloat16* base;  // first row of the unit
  int64_t ld, cols, col0, row0;
  int nrow;
};
__device__ __forceinline__ RowSrc rows_of(const EncAUnit& u) {
  const int64_t i0 = u.I * u.vb;
  return RowSrc{u.A + i0 * u.lda, u.lda, u.k, u.cx * kEncCols, i0,
                (int)(min(i0 + (int64_t)u.vb, u.m) - i0)};
}
__device__ __forceinline__ RowSrc rows_of(const EncBUnit& u) {
  const int64_t l0 = u.ry * kRowsPerCtaB;
  return RowSrc{u.B + l0 * u.ldb, u.ldb, u.n, u.cx * kEncCols, l0,
                (int)(min(l0 + (int64_t)kRowsPerCtaB, u.k) - l0)};
}

// FP8 E4M3 source of a single-problem pass (q == nullptr: the rows are bf16):
// the pass reads the e4m3 rows (8 bytes per lane per row), dequantises them
// with their 128 x 128 block scale, writes the exact values into the bf16
// operand plane the product reads, and forms the checksums from them -- one
// pass instead of a dequantisation pass and a checksum pass over the plane.
struct Fp8Src {
  const uint8_t* q;
  int64_t ldq;
  const float* sc;  // scale[row / 128][col / 128]
  int64_t sld;      // scale columns
  __nv_bfloat16* plane;
  int64_t pld;      // plane leading dimension (columns cols .. pld-1 are zero)
  int* inexact;     // set when a value is not exact in bf16
  // B pass of the native FP8 product: also write the codes transposed, B^T
  // (cols x ldbt bytes, zeros past the rows), or nullptr
  uint8_t* bt;
  int64_t ldbt;
};

// The B pass's transposed copy of a unit (128 rows x 256 columns of e4m3
// codes): each lane stores its 8 bytes of a row into a shared tile of 128 rows
// x 64 words, word column c of row r at c ^ (4 ((r / 16) % 8)), so that the
// transposing reads (16 consecutive rows of one word column, 8 row groups per
// warp) hit 32 distinct banks; then each thread turns 16 rows x 4 columns into
// four 16-byte pieces of rows of B^T (byte permutes), eight threads covering
// 128 contiguous bytes of a row.
constexpr int kBtBytes = 128 * 256;
__device__ __forceinline__ void bt_store_row(uint32_t* tileT, int t, int lane, uint2 raw) {
  const int s = ((t >> 4) & 7) << 2;
  *reinterpret_cast<uint2*>(&tileT[t * 64 + ((2 * lane) ^ s)]) = raw;
}

// A 4 x 4 byte block transposed: r0..r3 are four rows of four bytes; o[j] is
// column j (byte i from row i).
__device__ __forceinline__ void transpose4x4(uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3,
                                             uint32_t (&o)[4]) {
  const uint32_t lo01 = __byte_perm(r0, r1, 0x5140), hi01 = __byte_perm(r0, r1, 0x7362);
  const uint32_t lo23 = __byte_perm(r2, r3, 0x5140), hi23 = __byte_perm(r2, r3, 0x7362);
  o[0] = __byte_perm(lo01, lo23, 0x5410);
  o[1] = __byte_perm(lo01, lo23, 0x7632);
  o[2] = __byte_perm(hi01, hi23, 0x5410);
  o[3] = __byte_perm(hi01, hi23, 0x7632);
}

// Write a unit's tile (see bt_store_row) to B^T: B rows k0 .. (kvalid of them
// hold codes; the others are written as zeros), B columns n0 .. n0 + 255.
__device__ __forceinline__ void bt_write_unit(const uint32_t* tileT, uint8_t* __restrict__ Bt,
                                              int64_t ldbt, int64_t n, int64_t n0, int64_t k0,
                                              int kvalid) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int item = threadIdx.x + kThreads * h;
    const int kb = item & 7, ng = item >> 3;  // rows 16 kb .. +15, word column ng
    const int64_t ok = k0 + 16 * kb;
    uint32_t o[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t x[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = 16 * kb + 4 * q + i;
        x[i] = r < kvalid ? tileT[r * 64 + (ng ^ (kb << 2))] : 0u;
      }
      uint32_t y[4];
      transpose4x4(x[0], x[1], x[2], x[3], y);
#pragma unroll
      for (int j = 0; j < 4; ++j) o[j][q] = y[j];
    }
    if (ok < ldbt) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t on = n0 + 4 * ng + j;
        if (on < n)
          *reinterpret_cast<uint4*>(Bt + on * ldbt + ok) = make_uint4(o[j][0], o[j][1], o[j][2],
                                                                      o[j][3]);
      }
    }
  }
}


// Eight e4m3 values (w0, w1 little-endian) times scale: the fp32 values (zero
// from column cols on; `full`: all eight columns are below cols) and their bf16
// images.
__device__ __forceinline__ void dequant8(uint32_t w0, uint32_t w1, float scl, bool full,
                                         int64_t c0, int64_t cols, float (&v)[8],
                                         __nv_bfloat16 (&o)[8]) {
  const uint32_t w[2] = {w0, w1};
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const __half2_raw h2 = __nv_cvt_fp8x2_to_halfraw2(
        (__nv_fp8x2_storage_t)((w[t >> 1] >> (16 * (t & 1))) & 0xFFFFu), __NV_E4M3);
    const float2 f = __half22float2(__half2(h2));
    v[2 * t] = f.x * scl;
    v[2 * t + 1] = f.y * scl;
  }
  if (!full) {
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (c0 + q >= cols) v[q] = 0.f;
  }
#pragma unroll
  for (int q = 0; q < 8; q += 2) {
    const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[q], v[q + 1]);
    o[q] = b2.x;
    o[q + 1] = b2.y;
  }
}
// Every e4m3 value times `scl` is exact in bf16 (and in binary32) when the
// scale is +-0 or +-2^e with -117 <= e <= 119: the codes carry at most 4
// significant bits and lie between 2^-9 and 448 in magnitude, so the products
// stay normal.  Checked once per row and lane instead of per value.
__device__ __forceinline__ bool scale_exact(float scl) {
  const uint32_t b = __float_as_uint(scl), e = (b >> 23) & 0xFFu;
  return (b & 0x7FFFFFu) == 0u && ((e >= 10u && e <= 246u) || e == 0u);
}
// Any of the four e4m3 codes of w a NaN (S.1111.111)?
__device__ __forceinline__ bool nan_code4(uint32_t w) {
  return (((w & 0x7F7F7F7Fu) + 0x01010101u) & 0x80808080u) != 0u;
}
// Batches of kRowBatch rows of warp w (rows w + 8 j) in a unit of nrow rows.
__device__ __forceinline__ int warp_batches(int nrow, int warp) {
  const int nj = nrow > warp ? (nrow - warp + kEncWarps - 1) / kEncWarps : 0;
  return (nj + kRowBatch - 1) / kRowBatch;
}

// Unit lists: one problem (units in column-chunk-major order) or a group.
// A single problem's units go to the CTAs round-robin (at any time the CTAs
// stream neighbouring units); a group's go in contiguous runs, one per CTA, so
// that a CTA's consecutive units mostly belong to one problem and its table
// entries and problem record are in L1 when the next unit starts (round-robin,
// every unit of a CTA was another problem's, and its warps waited on those
// dependent loads at each unit).
struct SingleAUnits {
  static constexpr bool kChunked = false;
  EncAUnit base;
  int64_t ncx, cnt;
  __device__ __forceinline__ int64_t count() const { return cnt; }
  __device__ __forceinline__ EncAUnit get(int64_t u) const {
    EncAUnit x = base;
    x.cx = u % ncx;
    x.I = u / ncx;
    return x;
  }
};
struct SingleBUnits {
  static constexpr bool kChunked = false;
  EncBUnit base;
  int64_t ncx, cnt;
  __device__ __forceinline__ int64_t count() const { return cnt; }
  __device__ __forceinline__ EncBUnit get(int64_t u) const {
    EncBUnit x = base;
    x.cx = u % ncx;
    x.ry = u / ncx;
    return x;
  }
};
struct GroupAUnits {
  static constexpr bool kChunked = true;
  const GProb* probs;
  const int2* tab;
  int64_t cnt;
  __device__ __forceinline__ int64_t count() const { return cnt; }
  __device__ __forceinline__ EncAUnit get(int64_t u) const {
    const int2 e = tab[u];
    const GProb& P = probs[e.x];
    const int64_t ncx = cdiv(P.acs_ld, kEncCols);
    return EncAUnit{static_cast<const __nv_bfloat16*>(P.A), P.lda, P.m, P.k, kGrpVbR, kGrpEr,
                    static_cast<__nv_bfloat16*>(P.acs), P.acs_ld, P.rowpart, cdiv(P.k, 256),
                    P.partA, e.y % ncx, e.y / ncx};
  }
};
struct GroupBUnits {
  static constexpr bool kChunked = true;
  const GProb* probs;
  const int2* tab;
  int64_t cnt;
  __device__ __forceinline__ int64_t count() const { return cnt; }
  __device__ __forceinline__ EncBUnit get(int64_t u) const {
    const int2 e = tab[u];
    const GProb& P = probs[e.x];
    const int64_t ncx = cdiv(P.n, kEncCols);
    return EncBUnit{static_cast<const __nv_bfloat16*>(P.B), P.ldb, P.k, P.n, kGrpVbC, kGrpEc,
                    static_cast<__nv_bfloat16*>(P.bcs), P.bcs_ld, P.colpart, P.partB,
                    cdiv(P.k, kRowsPerCtaB), e.y % ncx, e.y / ncx};
  }
};

// The units of this CTA: first, first + step, ... below end.
struct UnitRange {
  int64_t first, end, step;
};
template <class Units>
__device__ __forceinline__ UnitRange unit_range(const Units& U) {
  if constexpr (Units::kChunked) {
    const int64_t per = cdiv(U.count(), (int64_t)gridDim.x);
    const int64_t f = (int64_t)blockIdx.x * per;
    return UnitRange{f, min(U.count(), f + per), 1};
  } else {
    return UnitRange{(int64_t)blockIdx.x, U.count(), (int64_t)gridDim.x};
  }
}

// A warp's copy cursor: issues the batches of the CTA's units in the order
// the arithmetic consumes them, one commit group per call (an empty group
// once nothing is left keeps the group count uniform).
template <class Units, bool kF8>
struct RingIssuer {
  using R = Ring<kF8>;
  const Units& U;
  const Fp8Src& f8;
  typename R::Slot* ring;
  int warp, lane;
  int64_t u, uend, ustep;
  int b, nbat, issued;
  RowSrc src;
  __device__ __forceinline__ void load() {
    if (u < uend) {
      src = rows_of(U.get(u));
      nbat = warp_batches(src.nrow, warp);
    }
  }
  __device__ __forceinline__ void start(const UnitRange& r) {
    u = r.first;
    uend = r.end;
    ustep = r.step;
    b = 0;
    issued = 0;
    nbat = 0;
    load();
  }
  __device__ __forceinline__ void next() {
    while (u < uend && b >= nbat) {
      u += ustep;
      b = 0;
      load();
    }
    if (u < uend) {
      typename R::Slot* slot = ring + (issued % R::kBatches) * kRowBatch * 32;
      const int64_t c0 = src.col0 + 8 * lane, rem = src.cols - c0;
      const uint32_t esz = kF8 ? 1u : 2u;  // bytes per element
      const uint32_t nb = rem >= 8 ? 8u * esz : (rem > 0 ? (uint32_t)rem * esz : 0u);
      // the batch's rows are kEncWarps apart: one pointer, advanced per row
      const int tb = warp + kEncWarps * b * kRowBatch;
      const uint32_t dst0 = static_cast<uint32_t>(__cvta_generic_to_shared(slot + lane));
      if constexpr (kF8) {
        const uint8_t* p = f8.q + (src.row0 + tb) * f8.ldq + c0;
        const int64_t step = kEncWarps * f8.ldq;
#pragma unroll
        for (int r = 0; r < kRowBatch; ++r, p += step) {
          const bool in = tb + kEncWarps * r < src.nrow && nb > 0;
          cp_async8(dst0 + r * 32 * (uint32_t)sizeof(typename R::Slot), in ? p : f8.q, in ? nb : 0u);
        }
      } else {
        const __nv_bfloat16* p = src.base + (int64_t)tb * src.ld + c0;
        const int64_t step = kEncWarps * src.ld;
#pragma unroll
        for (int r = 0; r < kRowBatch; ++r, p += step) {
          const bool in = tb + kEncWarps * r < src.nrow && nb > 0;
          cp_async16(dst0 + r * 32 * (uint32_t)sizeof(typename R::Slot), in ? p : src.base,
                     in ? nb : 0u);
        }
      }
      ++b;
    }
    cp_async_commit();
    ++issued;
  }
};

// Per-batch addressing of the e4m3 source: the scale index of the batch's
// first row (row0b: its row in the operand) and its plane row pointer; the
// batch's kRowBatch rows are kEncWarps apart, so they span fewer than 128 rows
// and at most two scale rows.
struct F8Batch {
  int64_t sidx;                // scale index of row row0b, column c0
  int rin;                     // row0b % 128
  __nv_bfloat16* plane;        // plane row row0b, column c0
  __device__ __forceinline__ F8Batch() : sidx(0), rin(0), plane(nullptr) {}
  __device__ __forceinline__ F8Batch(const Fp8Src& f8, int64_t row0b, int64_t c0)
      : sidx((row0b >> 7) * f8.sld + (c0 >> 7)),
        rin((int)(row0b & 127)),
        plane(f8.plane + row0b * f8.pld + c0) {}
};

// Row r of a batch from the ring: bf16 rows are unpacked; e4m3 rows are
// dequantised with their block scale, and their bf16 values written to the
// operand plane.
template <bool kF8>
__device__ __forceinline__ void ring_row(const typename Ring<kF8>::Slot& raw, const Fp8Src& f8,
                                         const F8Batch* fb, int r, bool valid, int64_t c0,
                                         int64_t cols, float (&v)[8], bool& bad) {
  if constexpr (kF8) {
    const bool in = valid && c0 < cols;
    const int64_t si = fb->sidx + (fb->rin + kEncWarps * r >= 128 ? f8.sld : 0);
    const float scl = in ? f8.sc[si] : 0.f;
    __nv_bfloat16 o[8];
    dequant8(raw.x, raw.y, scl, c0 + 8 <= cols, c0, cols, v, o);
    // a value that is not exact in bf16 (scale not a power of two in range)
    // or a NaN code (bytes past cols are zero-filled by the copy)
    bad |= in && (!scale_exact(scl) || nan_code4(raw.x) || nan_code4(raw.y));
    if (valid && c0 < f8.pld) store8(fb->plane + (int64_t)(kEncWarps * r) * f8.pld, o);
  } else {
    unpack8(raw, v);
  }
}

template <class Units, bool kF8>
__global__ void __launch_bounds__(kThreads, 2) k_encA_stream(const Units U, const Fp8Src f8) {
  __shared__ __align__(16) float red[kEncWarps * kEncCols * 2];
  __shared__ float sh[kThreads / 32];
  using R = Ring<kF8>;
  extern __shared__ uint4 ring_s[];  // R::kBytes
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  typename R::Slot* ring =
      reinterpret_cast<typename R::Slot*>(ring_s) + warp * R::kBatches * kRowBatch * 32;
  bool bad = false;
  RingIssuer<Units, kF8> is{U, f8, ring, warp, lane};
  const UnitRange ur = unit_range(U);
  is.start(ur);
#pragma unroll
  for (int i = 0; i < R::kBatches; ++i) is.next();
  constexpr int kLanesPerRow = 32 / kRowBatch;
  int consumed = 0;
  for (int64_t u = ur.first; u < ur.end; u += ur.step) {
    const EncAUnit X = U.get(u);
    const RowSrc src = rows_of(X);
    const int nbat = warp_batches(src.nrow, warp);
    const float sc = scalbnf(1.0f, -X.e);
    float se[8], sw[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) se[q] = sw[q] = 0.f;
    for (int b = 0; b < nbat; ++b) {
      cp_async_wait<R::kBatches - 1>();  // this warp's oldest batch has landed
      const typename R::Slot* slot = ring + (consumed % R::kBatches) * kRowBatch * 32;
      float sq[kRowBatch];
      const int tb = warp + kEncWarps * b * kRowBatch;
      const int64_t c0 = src.col0 + 8 * lane;
      F8Batch fb = kF8 ? F8Batch(f8, src.row0 + tb, c0) : F8Batch();
#pragma unroll
      for (int r = 0; r < kRowBatch; ++r) {
        const int t = tb + kEncWarps * r;
        float v[8];
        ring_row<kF8>(slot[r * 32 + lane], f8, &fb, r, t < src.nrow, c0, src.cols, v, bad);
        lpA_rows(v, t, sc, se, sw, sq[r]);
      }
      ++consumed;
      is.next();  // refills the slot just read (each lane reads only its own copies)
      reduce_rows<kRowBatch>(sq, lane);
      const int t = warp + kEncWarps * (b * kRowBatch + lane / kLanesPerRow);
      if (lane % kLanesPerRow == 0 && t < src.nrow)
        X.rowpart[(X.I * X.vb + t) * X.nchr + X.cx] = sq[0];
    }
    lpA_finish(se, sw, X.acs, X.ldk, X.part, X.nchr, X.cx, X.I, red, sh);
  }
  cp_async_wait<0>();
  if (kF8 && bad) atomicExch(f8.inexact, 1);
}

template <class Units, bool kF8>
__global__ void __launch_bounds__(kThreads, 2) k_encB_stream(const Units U, const Fp8Src f8) {
  __shared__ __align__(16) float red[kEncWarps * kEncCols];
  __shared__ float redq[kEncWarps * 32 * 2];
  using R = Ring<kF8>;
  extern __shared__ uint4 ring_s[];  // R::kBytes (+ kBtBytes for e4m3: the B^T tile)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  typename R::Slot* ring =
      reinterpret_cast<typename R::Slot*>(ring_s) + warp * R::kBatches * kRowBatch * 32;
  uint32_t* tileT = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(ring_s) + R::kBytes);
  const bool wbt = kF8 && f8.bt != nullptr;  // this pass also writes B^T
  bool bad = false;
  RingIssuer<Units, kF8> is{U, f8, ring, warp, lane};
  const UnitRange ur = unit_range(U);
  is.start(ur);
#pragma unroll
  for (int i = 0; i < R::kBatches; ++i) is.next();
  int consumed = 0;
  for (int64_t u = ur.first; u < ur.end; u += ur.step) {
    const EncBUnit X = U.get(u);
    const RowSrc src = rows_of(X);
    const int nbat = warp_batches(src.nrow, warp);
    const int64_t c0 = X.cx * kEncCols + 8 * lane, l0 = X.ry * kRowsPerCtaB;
    const int seg = X.vb / 8;  // lanes per verify block (1 .. 32)
    const bool leader = (lane % seg) == 0 && c0 < X.n;
    const int64_t J = c0 / X.vb;
    const float sc = scalbnf(1.0f, -X.e);
    float wq[8], cs[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      wq[q] = (float)((int)((c0 + q) % X.vb) + 1) * sc;
      cs[q] = 0.f;
    }
    float q0 = 0.f, q1 = 0.f;
    for (int b = 0; b < nbat; ++b) {
      cp_async_wait<R::kBatches - 1>();
      const typename R::Slot* slot = ring + (consumed % R::kBatches) * kRowBatch * 32;
      if (seg == 32) {
        // one verify block across the warp: the batch's 8 rows' (e, w) sums
        // reduce in one transposing butterfly (15 + 1 shuffles for 16 sums);
        // lane l then holds sum l / 2: row l / 4, e (l / 2 even) or w
        float sums[2 * kRowBatch];
        const int tb = warp + kEncWarps * b * kRowBatch;
        F8Batch fb = kF8 ? F8Batch(f8, l0 + tb, c0) : F8Batch();
#pragma unroll
        for (int r = 0; r < kRowBatch; ++r) {
          const int t = tb + kEncWarps * r;
          float v[8];
          ring_row<kF8>(slot[r * 32 + lane], f8, &fb, r, t < src.nrow, c0, X.n, v, bad);
          if constexpr (kF8)
            if (wbt) bt_store_row(tileT, t, lane, slot[r * 32 + lane]);
          lpB_row(v, wq, cs, sums[2 * r], sums[2 * r + 1]);
        }
        ++consumed;
        is.next();
        reduce_rows<2 * kRowBatch>(sums, lane);
        const int t = warp + kEncWarps * (b * kRowBatch + (lane >> 2)), kind = (lane >> 1) & 1;
        if ((lane & 1) == 0 && t < src.nrow && X.cx * kEncCols < X.n) {
          __nv_bfloat16 pc[2];
          split(sums[0], pc[0], pc[1]);
          *reinterpret_cast<uint32_t*>(X.bcs + (l0 + t) * X.ldcs + 4 * J + 2 * kind) =
              *reinterpret_cast<const uint32_t*>(pc);
          if (kind)
            q1 = fmaf(sums[0], sums[0], q1);
          else
            q0 = fmaf(sums[0], sums[0], q0);
        }
      } else {
        const int tb = warp + kEncWarps * b * kRowBatch;
        F8Batch fb = kF8 ? F8Batch(f8, l0 + tb, c0) : F8Batch();
#pragma unroll
        for (int r = 0; r < kRowBatch; ++r) {
          const int t = tb + kEncWarps * r;
          float v[8], se, sw;
          ring_row<kF8>(slot[r * 32 + lane], f8, &fb, r, t < src.nrow, c0, X.n, v, bad);
          if constexpr (kF8)
            if (wbt) bt_store_row(tileT, t, lane, slot[r * 32 + lane]);
          lpB_row(v, wq, cs, se, sw);
          lpB_store_shfl(se, sw, seg, leader, t < src.nrow, X.bcs + (l0 + t) * X.ldcs + 4 * J,
                         q0, q1);
        }
        ++consumed;
        is.next();
      }
    }
    if (seg == 32) {  // the checksum-norm partials of the warp's rows to lane 0
      q0 = warp_sumf(q0);
      q1 = warp_sumf(q1);
    }
    lpB_finish(cs, q0, q1, X.n, X.vb, X.colpart, X.part, X.nch, X.cx, X.ry, red, redq);
    if (wbt) {  // every warp's rows of the unit are in the tile (lpB_finish synchronised)
      bt_write_unit(tileT, f8.bt, f8.ldbt, X.n, X.cx * kEncCols, l0, src.nrow);
      __syncthreads();  // the tile is rewritten by the next unit
    }
  }
  cp_async_wait<0>();
  if (kF8 && bad) atomicExch(f8.inexact, 1);
}

// The same outputs for any verify block size (one warp per row segment).
__global__ void __launch_bounds__(kThreads) k_lpB_rows_any(const __nv_bfloat16* __restrict__ B,
                                                           int64_t ldb, int64_t k, int64_t n,
                                                           int vb, int e,
                                                           __nv_bfloat16* __restrict__ bcs,
                                                           int64_t ldcs,
                                                           double* __restrict__ part,
                                                           int64_t nch) {
  const int lane = threadIdx.x & 31;
  const int64_t chunk = (int64_t)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
  if (chunk >= nch) return;
  const int64_t nvb = cdiv(n, vb);
  const float sc = scalbnf(1.0f, -e);
  for (int64_t J = blockIdx.y; J < nvb; J += gridDim.y) {
    const int64_t j0 = J * vb, j1 = min(j0 + (int64_t)vb, n);
    const int64_t l0 = chunk * kRowsPerCtaB, l1 = min(l0 + kRowsPerCtaB, k);
    float q0 = 0.f, q1 = 0.f;
    for (int64_t l = l0; l < l1; ++l) {
      float se = 0.f, sw = 0.f;
      for (int64_t j = j0 + lane; j < j1; j += 32) {
        const float b = ldf(B + l * ldb + j);
        se += b;
        sw = fmaf((float)(j - j0 + 1) * sc, b, sw);
      }
      se = warp_sumf(se);
      sw = warp_sumf(sw);
      if (lane == 0) {
        __nv_bfloat16 h, lo;
        split(se, h, lo);
        bcs[l * ldcs + 4 * J + 0] = h;
        bcs[l * ldcs + 4 * J + 1] = lo;
        split(sw, h, lo);
        bcs[l * ldcs + 4 * J + 2] = h;
        bcs[l * ldcs + 4 * J + 3] = lo;
      }
      q0 = fmaf(se, se, q0);
      q1 = fmaf(sw, sw, q1);
    }
    if (lane == 0) {
      part[(2 * J) * nch + chunk] = q0;
      part[(2 * J + 1) * nch + chunk] = q1;
    }
  }
}

// Column partial sums of squares for the generic path.  Grid (ceil(n/256), nch).
__global__ void __launch_bounds__(kThreads) k_lp_col_sq(const __nv_bfloat16* __restrict__ B,
                                                        int64_t ldb, int64_t k, int64_t n,
                                                        float* __restrict__ colpart) {
  const int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (j >= n) return;
  const int64_t nch = cdiv(k, kRowsPerCtaB);
  for (int64_t c = blockIdx.y; c < nch; c += gridDim.y) {
    const int64_t l0 = c * kRowsPerCtaB, l1 = min(l0 + kRowsPerCtaB, k);
    float s = 0.f;
    for (int64_t l = l0; l < l1; ++l) {
      const float b = ldf(B + l * ldb + j);
      s = fmaf(b, b, s);
    }
    colpart[c * n + j] = s;
  }
}

// The line norms and the threshold norms of their verify blocks in one pass:
// CTA I (256 threads) takes the lines of verify block I, each line's norm
// sqrt(sum_c part[t so + c sc]) from its fp32 partials (summed in fp32: the
// norms scale the thresholds, a few u32 of relative error is immaterial), then
// the block's norms: sqrt of the sums of squares of its line norms, unweighted
// and weighted (the weights of the block's lines), and of its checksum partials.
__global__ void __launch_bounds__(kThreads) k_lp_norms_blk(
    const float* __restrict__ part, int64_t nout, int64_t nch, int64_t so, int64_t sc,
    double* __restrict__ nvec, int vb, int e, const double* __restrict__ cpart, int64_t cnch,
    double* __restrict__ nblk) {
  __shared__ float sh[kThreads / 32];
  const int64_t I = blockIdx.x;
  const int64_t t0 = I * vb, t1 = min(t0 + (int64_t)vb, nout);
  const float scw = scalbnf(1.0f, -e);
  float f0 = 0.f, f1 = 0.f;
  for (int64_t t = t0 + threadIdx.x; t < t1; t += kThreads) {
    float s[4] = {0.f, 0.f, 0.f, 0.f};
    int64_t c = 0;
    for (; c + 4 <= nch; c += 4) {
#pragma unroll
      for (int j = 0; j < 4; ++j) s[j] += part[t * so + (c + j) * sc];
    }
    for (; c < nch; ++c) s[0] += part[t * so + c * sc];
    const float v = sqrtf((s[0] + s[1]) + (s[2] + s[3]));
    nvec[t] = (double)v;
    const float wv = (float)(t - t0 + 1) * scw * v;
    f0 = fmaf(v, v, f0);
    f1 = fmaf(wv, wv, f1);
  }
  float q0 = 0.f, q1 = 0.f;
  for (int64_t c = threadIdx.x; c < cnch; c += kThreads) {
    q0 += (float)cpart[(2 * I) * cnch + c];
    q1 += (float)cpart[(2 * I + 1) * cnch + c];
  }
  f0 = block_sumf(f0, sh);
  f1 = block_sumf(f1, sh);
  q0 = block_sumf(q0, sh);
  q1 = block_sumf(q1, sh);
  if (threadIdx.x == 0) {
    nblk[4 * I + 0] = (double)sqrtf(f0);
    nblk[4 * I + 1] = (double)sqrtf(f1);
    nblk[4 * I + 2] = (double)sqrtf(q0);
    nblk[4 * I + 3] = (double)sqrtf(q1);
  }
}

// ---------------- split bf16x3 (binary32 inputs)

// Eight consecutive binary32 elements starting at column c (zeros past len).
__device__ __forceinline__ void load8f(const float* row, int64_t c, int64_t len, float (&v)[8]) {
  if (c + 8 <= len && ((reinterpret_cast<uintptr_t>(row + c) & 15) == 0)) {
    const float4 a = *reinterpret_cast<const float4*>(row + c);
    const float4 b = *reinterpret_cast<const float4*>(row + c + 4);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  } else {
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = (c + q < len) ? row[c + q] : 0.f;
  }
}

// The bf16 planes of a split operand: x = p[0] + p[1] (+ p[2]) with
// p[i] = bf16 of what the earlier pieces leave (each difference is exact in
// fp32); np = 2 (bf16x3) or 3 (bf16x6).
struct Planes {
  __nv_bfloat16* p[3];
  int np;
};

__device__ __forceinline__ void split_pieces(float x, __nv_bfloat16 (&out)[3]) {
  float r = x;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    out[i] = __float2bfloat16_rn(r);
    r -= __bfloat162float(out[i]);
  }
}

// One element into the planes at offset off.
__device__ __forceinline__ void store_split1(const Planes& P, int64_t off, float x) {
  __nv_bfloat16 h[3];
  split_pieces(x, h);
#pragma unroll
  for (int i = 0; i < 3; ++i)
    if (i < P.np) P.p[i][off] = h[i];
}

// Eight consecutive values into the planes at offset off (16-byte stores).
__device__ __forceinline__ void store_split8(const Planes& P, int64_t off, const float (&v)[8]) {
  __nv_bfloat16 h[3][8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    __nv_bfloat16 t[3];
    split_pieces(v[q], t);
#pragma unroll
    for (int i = 0; i < 3; ++i) h[i][q] = t[i];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
    if (i < P.np) store8(P.p[i] + off, h[i]);
}

// Rows of binary32 loads a thread of the split passes issues ahead.
constexpr int kSplitRows = 8;

// A: planes (m x ldk), column checksums of A per verify block from the
// binary32 values (rows 2I, 2I+1 of the acs planes), per-row partial sums of
// squares and checksum-norm partials.  CTA = 2048 columns x a block.
__global__ void __launch_bounds__(kThreads) k_x3A_cols(const float* __restrict__ A, int64_t lda,
                                                       int64_t m, int64_t k, int vb, int e,
                                                       const Planes op, const Planes cs,
                                                       int64_t ldk, float* __restrict__ rowpart,
                                                       int64_t nchr, double* __restrict__ part,
                                                       int64_t nch, int cs_on) {
  __shared__ float sh[kThreads / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t c0 = (int64_t)blockIdx.x * kColsPerCta + 8 * threadIdx.x;
  const int64_t nvb = cdiv(m, vb);
  const float sc = scalbnf(1.0f, -e);
  for (int64_t I = blockIdx.y; I < nvb; I += gridDim.y) {
    const int64_t i0 = I * vb, i1 = min(i0 + (int64_t)vb, m);
    float se[8], sw[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) se[q] = sw[q] = 0.f;
    // kSplitRows rows' loads in flight per thread before the first of them is used
    // (the plane stores would otherwise hold each next row's loads back)
    for (int64_t ib = i0; ib < i1; ib += kSplitRows) {
      float vb8[kSplitRows][8];
#pragma unroll
      for (int r = 0; r < kSplitRows; ++r)
        if (ib + r < i1) load8f(A + (ib + r) * lda, c0, k, vb8[r]);
#pragma unroll
      for (int r = 0; r < kSplitRows; ++r) {
        const int64_t i = ib + r;
        if (i >= i1) break;
        const float (&v)[8] = vb8[r];
        if (c0 < ldk) store_split8(op, i * ldk + c0, v);
        const float w = (float)(int)(i - i0 + 1) * sc;
        float sq = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          se[q] += v[q];
          sw[q] = fmaf(w, v[q], sw[q]);
          sq = fmaf(v[q], v[q], sq);
        }
        sq = warp_sumf(sq);
        const int64_t rc = (int64_t)blockIdx.x * (kThreads / 32) + warp;
        if (lane == 0 && rc < nchr) rowpart[i * nchr + rc] = sq;
      }
    }
    if (!cs_on) continue;  // chained: the checksum rows are carried, not formed
    float q0 = 0.f, q1 = 0.f;
    if (c0 < ldk) {
      store_split8(cs, (2 * I) * ldk + c0, se);
      store_split8(cs, (2 * I + 1) * ldk + c0, sw);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        q0 = fmaf(se[q], se[q], q0);
        q1 = fmaf(sw[q], sw[q], q1);
      }
    }
    const float t0 = block_sumf(q0, sh);
    if (threadIdx.x == 0) part[(2 * I) * nch + blockIdx.x] = (double)t0;
    const float t1 = block_sumf(q1, sh);
    if (threadIdx.x == 0) part[(2 * I + 1) * nch + blockIdx.x] = (double)t1;
  }
}

// Block checksum rows S^(c)[t] = sum_I c_{c,I} A[I*bs + t] (c < f) into rows
// 2 nvr + c*bs + t of the planes (cs points at row 2 nvr of each plane).
__global__ void __launch_bounds__(kThreads) k_x3A_block(const float* __restrict__ A, int64_t lda,
                                                        int64_t k, int p, int64_t bs, int f,
                                                        const Planes cs, int64_t ldk) {
  const int64_t l = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (l >= k) return;
  for (int64_t ct = blockIdx.y; ct < f * bs; ct += gridDim.y) {
    const int c = (int)(ct / bs);
    const int64_t t = ct - c * bs;
    float s = 0.f;
    for (int I = 0; I < p; ++I) s = fmaf((float)block_coef(c, I, p), A[(I * bs + t) * lda + l], s);
    store_split1(cs, ct * ldk + l, s);
  }
}

// B: planes (k x ldn), row checksums per verify column block (columns 2J,
// 2J+1 of the bcs planes), per-column partial sums of squares and
// checksum-norm partials.  Verify blocks of 8 .. 256 columns (power of two).
__global__ void __launch_bounds__(kThreads) k_x3B_rows(const float* __restrict__ B, int64_t ldb,
                                                       int64_t k, int64_t n, int vb, int e,
                                                       const Planes op, int64_t ldn,
                                                       const Planes cs, int64_t ldcs,
                                                       float* __restrict__ colpart,
                                                       double* __restrict__ part, int64_t nch) {
  const int lane = threadIdx.x & 31;
  const int64_t c0 = (int64_t)blockIdx.x * kColsPerCta + 8 * threadIdx.x;
  const int64_t l0 = (int64_t)blockIdx.y * kRowsPerCtaB, l1 = min(l0 + kRowsPerCtaB, k);
  const int seg = vb / 8;
  const bool leader = (lane % seg) == 0 && c0 < n;
  const int64_t J = c0 / vb;
  const float sc = scalbnf(1.0f, -e);
  float wq[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) wq[q] = (float)((int)((c0 + q) % vb) + 1) * sc;
  float cs2[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) cs2[q] = 0.f;
  float q0 = 0.f, q1 = 0.f;
  for (int64_t lb = l0; lb < l1; lb += kSplitRows) {
    float vb8[kSplitRows][8];  // the rows' loads in flight before the first is used
#pragma unroll
    for (int r = 0; r < kSplitRows; ++r)
      if (lb + r < l1) load8f(B + (lb + r) * ldb, c0, n, vb8[r]);
#pragma unroll
    for (int r = 0; r < kSplitRows; ++r) {
      const int64_t l = lb + r;
      if (l >= l1) break;
      const float (&v)[8] = vb8[r];
      if (c0 < ldn) store_split8(op, l * ldn + c0, v);
      float se = 0.f, sw = 0.f;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        se += v[q];
        sw = fmaf(wq[q], v[q], sw);
        cs2[q] = fmaf(v[q], v[q], cs2[q]);
      }
      for (int o = seg >> 1; o > 0; o >>= 1) {
        se += __shfl_xor_sync(0xffffffffu, se, o);
        sw += __shfl_xor_sync(0xffffffffu, sw, o);
      }
      if (leader) {
        store_split1(cs, l * ldcs + 2 * J, se);
        store_split1(cs, l * ldcs + 2 * J + 1, sw);
        q0 = fmaf(se, se, q0);
        q1 = fmaf(sw, sw, q1);
      }
    }
  }
  if (leader) {
    part[(2 * J) * nch + blockIdx.y] = q0;
    part[(2 * J + 1) * nch + blockIdx.y] = q1;
  }
#pragma unroll
  for (int q = 0; q < 8; ++q)
    if (c0 + q < n) colpart[blockIdx.y * n + c0 + q] = cs2[q];
}

// Any verify block size: planes and column partials by one kernel, row
// checksums by one warp per (J, 128 rows).
__global__ void __launch_bounds__(kThreads) k_x3B_split(const float* __restrict__ B, int64_t ldb,
                                                        int64_t k, int64_t n, const Planes op,
                                                        int64_t ldn, float* __restrict__ colpart) {
  const int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (j >= ldn) return;
  const int64_t nch = cdiv(k, kRowsPerCtaB);
  for (int64_t c = blockIdx.y; c < nch; c += gridDim.y) {
    const int64_t l0 = c * kRowsPerCtaB, l1 = min(l0 + kRowsPerCtaB, k);
    float s = 0.f;
    for (int64_t l = l0; l < l1; ++l) {
      const float b = j < n ? B[l * ldb + j] : 0.f;
      store_split1(op, l * ldn + j, b);
      s = fmaf(b, b, s);
    }
    if (j < n) colpart[c * n + j] = s;
  }
}

__global__ void __launch_bounds__(kThreads) k_x3B_rows_any(const float* __restrict__ B,
                                                           int64_t ldb, int64_t k, int64_t n,
                                                           int vb, int e, const Planes cs,
                                                           int64_t ldcs,
                                                           double* __restrict__ part,
                                                           int64_t nch) {
  const int lane = threadIdx.x & 31;
  const int64_t chunk = (int64_t)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
  if (chunk >= nch) return;
  const int64_t nvb = cdiv(n, vb);
  const float sc = scalbnf(1.0f, -e);
  for (int64_t J = blockIdx.y; J < nvb; J += gridDim.y) {
    const int64_t j0 = J * vb, j1 = min(j0 + (int64_t)vb, n);
    const int64_t l0 = chunk * kRowsPerCtaB, l1 = min(l0 + kRowsPerCtaB, k);
    float q0 = 0.f, q1 = 0.f;
    for (int64_t l = l0; l < l1; ++l) {
      float se = 0.f, sw = 0.f;
      for (int64_t j = j0 + lane; j < j1; j += 32) {
        const float b = B[l * ldb + j];
        se += b;
        sw = fmaf((float)(int)(j - j0 + 1) * sc, b, sw);
      }
      se = warp_sumf(se);
      sw = warp_sumf(sw);
      if (lane == 0) {
        store_split1(cs, l * ldcs + 2 * J, se);
        store_split1(cs, l * ldcs + 2 * J + 1, sw);
      }
      q0 = fmaf(se, se, q0);
      q1 = fmaf(sw, sw, q1);
    }
    if (lane == 0) {
      part[(2 * J) * nch + chunk] = q0;
      part[(2 * J + 1) * nch + chunk] = q1;
    }
  }
}

// E[r][j] = sum_{p < npc} E16[npc r + p][j]: the products of the npc pieces of
// each checksum row (bf16: hi and lo rows, npc = 2; split bf16x3: npc = 1),
// added in binary64.
__global__ void k_fold_E(const float* __restrict__ E16, int64_t R, int npc, int64_t n,
                         double* __restrict__ E) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  for (int64_t r = blockIdx.y; r < R; r += gridDim.y) {
    double v = 0.0;
    for (int p = 0; p < npc; ++p) v += (double)E16[(npc * r + p) * n + j];
    E[r * n + j] = v;
  }
}

// F[i][c] = sum_{p < npc} F16[i][npc c + p]   (binary64)
__global__ void k_fold_F(const float* __restrict__ F16, int64_t m, int64_t Cc, int64_t C16,
                         int npc, double* __restrict__ F) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m * Cc) return;
  const int64_t i = t / Cc, c = t % Cc;
  double v = 0.0;
  for (int p = 0; p < npc; ++p) v += (double)F16[i * C16 + npc * c + p];
  F[i * Cc + c] = v;
}

// ---------------- FP8 E4M3 with binary32 block scales

// Dequantised operand plane: out[i][j] = e4m3(q[i][j]) * scale[i/128][j/128]
// as bf16, which is exact when the scales are powers of two (an e4m3 value has
// at most 4 significant bits).  A value that bf16 cannot hold exactly sets
// *inexact (the call then reports ABFT_ERR_INVALID); columns cols .. ld-1 of
// the plane are zero.  Thread = 8 consecutive elements (one 8-byte load, one
// 16-byte store) of kDqRows rows, whose loads are in flight together; the 8
// elements share one scale (8 divides 128).
constexpr int kDqRows = 8;

__global__ void __launch_bounds__(kThreads) k_fp8_dequant(const uint8_t* __restrict__ q, int64_t ldq,
                                                          int64_t rows, int64_t cols,
                                                          const float* __restrict__ scale,
                                                          __nv_bfloat16* __restrict__ out,
                                                          int64_t ld, int* inexact) {
  const int64_t c0 = 8 * ((int64_t)blockIdx.x * kThreads + threadIdx.x);
  if (c0 >= ld) return;
  const int64_t sld = cdiv(cols, 128);
  const bool full8 = c0 + 8 <= cols;
  bool bad = false;
  for (int64_t i0 = (int64_t)blockIdx.y * kDqRows; i0 < rows; i0 += (int64_t)gridDim.y * kDqRows) {
    uint2 raw[kDqRows];
    float sc[kDqRows];
#pragma unroll
    for (int r = 0; r < kDqRows; ++r) {
      const int64_t i = i0 + r;
      raw[r] = make_uint2(0u, 0u);
      sc[r] = 0.f;
      if (i < rows && c0 < cols) {
        const uint8_t* p = q + i * ldq + c0;
        if (full8 && (reinterpret_cast<uintptr_t>(p) & 7) == 0) {
          raw[r] = *reinterpret_cast<const uint2*>(p);
        } else {
          uint32_t w[2] = {0u, 0u};
          for (int t = 0; t < 8; ++t)
            if (c0 + t < cols) w[t >> 2] |= (uint32_t)p[t] << (8 * (t & 3));
          raw[r] = make_uint2(w[0], w[1]);
        }
        sc[r] = scale[(i / 128) * sld + c0 / 128];
      }
    }
#pragma unroll
    for (int r = 0; r < kDqRows; ++r) {
      const int64_t i = i0 + r;
      if (i >= rows) break;
      const uint32_t w[2] = {raw[r].x, raw[r].y};
      __nv_bfloat16 o[8];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const __half2_raw h2 = __nv_cvt_fp8x2_to_halfraw2(
            (__nv_fp8x2_storage_t)((w[t >> 1] >> (16 * (t & 1))) & 0xFFFFu), __NV_E4M3);
        const float2 f = __half22float2(__half2(h2));
        const float v0 = c0 + 2 * t < cols ? f.x * sc[r] : 0.f;
        const float v1 = c0 + 2 * t + 1 < cols ? f.y * sc[r] : 0.f;
        o[2 * t] = __float2bfloat16_rn(v0);
        o[2 * t + 1] = __float2bfloat16_rn(v1);
      }
      // the same rule as the streaming passes (bytes past cols are zero here)
      bad |= c0 < cols && (!scale_exact(sc[r]) || nan_code4(w[0]) || nan_code4(w[1]));
      store8(out + i * ld + c0, o);
    }
  }
  if (bad) atomicExch(inexact, 1);
}

// ---------------- chained split products (binary32 operands)
// A chained bf16x3 / bf16x6 product carries the earlier product's binary64
// checksums (section 3.2); they enter the checksum planes as bf16 pieces of
// the binary64 values (three pieces hold a value to 2^-27, two to 2^-18 --
// the representation the thresholds already carry as u_cs).

__device__ __forceinline__ void split_pieces_d(double x, __nv_bfloat16 (&out)[3]) {
  double r = x;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    out[i] = __double2bfloat16(r);
    r -= (double)__bfloat162float(out[i]);
  }
}

// Carried rows E[r][l] (rows x k, binary64, ld k) into row r of the checksum
// planes (ld ldk; columns k .. ldk-1 zero), and partials of the squared norms
// of the first nrm rows: part[r * nch + chunk], chunks of 8 * 256 columns
// (the layout the split A pass leaves).  Grid (nch, <= 65535); thread = 8
// consecutive columns.
__global__ void __launch_bounds__(kThreads) k_carried_rows_split(const double* __restrict__ E,
                                                                 int64_t rows, int64_t k,
                                                                 const Planes cs, int64_t ldk,
                                                                 double* __restrict__ part,
                                                                 int64_t nch, int64_t nrm) {
  __shared__ double shd[kThreads / 32];
  const int64_t c0 = (int64_t)blockIdx.x * kColsPerCta + 8 * threadIdx.x;
  for (int64_t r = blockIdx.y; r < rows; r += gridDim.y) {
    double q = 0.0;
    if (c0 < ldk) {
      __nv_bfloat16 h[3][8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const double x = c0 + t < k ? E[r * k + c0 + t] : 0.0;
        q = fma(x, x, q);
        __nv_bfloat16 pc[3];
        split_pieces_d(x, pc);
#pragma unroll
        for (int i = 0; i < 3; ++i) h[i][t] = pc[i];
      }
#pragma unroll
      for (int i = 0; i < 3; ++i)
        if (i < cs.np) store8(cs.p[i] + r * ldk + c0, h[i]);
    }
    if (r < nrm) {  // uniform in the block
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
      __syncthreads();
      if ((threadIdx.x & 31) == 0) shd[threadIdx.x >> 5] = q;
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += shd[w];
        part[r * nch + blockIdx.x] = t;
      }
    }
  }
}

// Carried columns F[l][c] (k x Cc, binary64) into column c of the checksum
// planes (ld ldcs), and partials part[c * nch + chunk] of their squared norms
// over chunks of 128 rows (the layout the split B pass leaves).  One thread
// per (column, chunk).
__global__ void __launch_bounds__(kThreads) k_carried_cols_split(const double* __restrict__ F,
                                                                 int64_t k, int64_t Cc,
                                                                 const Planes cs, int64_t ldcs,
                                                                 double* __restrict__ part,
                                                                 int64_t nch) {
  const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (t >= Cc * nch) return;
  const int64_t c = t % Cc, chunk = t / Cc;
  const int64_t l0 = chunk * kRowsPerCtaB, l1 = min(l0 + (int64_t)kRowsPerCtaB, k);
  double q = 0.0;
  for (int64_t l = l0; l < l1; ++l) {
    const double x = F[l * Cc + c];
    q = fma(x, x, q);
    __nv_bfloat16 pc[3];
    split_pieces_d(x, pc);
#pragma unroll
    for (int i = 0; i < 3; ++i)
      if (i < cs.np) cs.p[i][l * ldcs + c] = pc[i];
  }
  part[c * nch + chunk] = q;
}

unsigned gy(int64_t v) { return (unsigned)(v < 65535 ? v : 65535); }

// The streaming passes keep their row rings in dynamic shared memory beyond
// the default 48 KiB.
template <class Units, bool kF8 = false>
cudaError_t launch_stream_A(const Units& U, cudaStream_t st, const Fp8Src& f8 = Fp8Src{}) {
  cudaError_t e = cudaFuncSetAttribute(k_encA_stream<Units, kF8>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       Ring<kF8>::kBytes);
  if (e != cudaSuccess || U.cnt == 0) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t grid = std::min<int64_t>(U.cnt, 2 * (int64_t)std::max(sms, 1));  // 2 CTAs per SM
  k_encA_stream<Units, kF8><<<(unsigned)grid, kThreads, Ring<kF8>::kBytes, st>>>(U, f8);
  count_launches(1);
  return cudaGetLastError();
}
template <class Units, bool kF8 = false>
cudaError_t launch_stream_B(const Units& U, cudaStream_t st, const Fp8Src& f8 = Fp8Src{}) {
  constexpr int kSmem = Ring<kF8>::kBytes + (kF8 ? kBtBytes : 0);
  cudaError_t e = cudaFuncSetAttribute(k_encB_stream<Units, kF8>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
  if (e != cudaSuccess || U.cnt == 0) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t grid = std::min<int64_t>(U.cnt, 2 * (int64_t)std::max(sms, 1));
  k_encB_stream<Units, kF8><<<(unsigned)grid, kThreads, kSmem, st>>>(U, f8);
  count_launches(1);
  return cudaGetLastError();
}

// B^T of the e4m3 codes (the K-major B operand of the product's native FP8
// data tiles): B is k x n (ldb bytes, 16-byte aligned rows), Bt is n x ldbt
// (ldbt = ceil16(k); the bytes past k are written as zero).  A CTA moves a
// 128 x 128 byte tile: 16-byte row loads into shared memory (4-byte words,
// the word column XOR-ed with 4 x (row / 16) so the transposing reads hit 32
// distinct banks), then each thread transposes a 16 (k) x 4 (n) byte block in
// registers (byte permutes) and stores four 16-byte pieces of rows of B^T
// (eight threads cover 128 contiguous bytes of a row).  Grid (ceil(n/128),
// min(ceil(ldbt/128), 65535)).
__global__ void __launch_bounds__(256) k_transpose_u8(const uint8_t* __restrict__ B, int64_t ldb,
                                                      int64_t k, int64_t n,
                                                      uint8_t* __restrict__ Bt, int64_t ldbt) {
  __shared__ __align__(16) uint32_t tile[128][32];
  const int t = threadIdx.x;
  const int kb = t & 7, w = t >> 3;  // transpose: k rows 16 kb .. +15, n bytes 4 w .. +3
  const int64_t n0 = (int64_t)blockIdx.x * 128;
  for (int64_t k0 = (int64_t)blockIdx.y * 128; k0 < ldbt; k0 += (int64_t)gridDim.y * 128) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = t + 256 * q, r = idx >> 3, c = (idx & 7) * 4;
      const int64_t kk = k0 + r, nn = n0 + 4 * c;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (kk < k) {
        if (nn + 16 <= n) {
          v = *reinterpret_cast<const uint4*>(B + kk * ldb + nn);
        } else {
          uint32_t x[4] = {0u, 0u, 0u, 0u};
          for (int i = 0; i < 16; ++i)
            if (nn + i < n) x[i >> 2] |= (uint32_t)B[kk * ldb + nn + i] << (8 * (i & 3));
          v = make_uint4(x[0], x[1], x[2], x[3]);
        }
      }
      *reinterpret_cast<uint4*>(&tile[r][c ^ (((r >> 4) & 7) << 2)]) = v;
    }
    __syncthreads();
    uint32_t o[4][4];  // o[j][q]: row n = 4 w + j of B^T, k bytes 16 kb + 4 q .. +3
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = 16 * kb + 4 * q, col = w ^ (kb << 2);
      uint32_t x[4];
      transpose4x4(tile[r][col], tile[r + 1][col], tile[r + 2][col], tile[r + 3][col], x);
#pragma unroll
      for (int j = 0; j < 4; ++j) o[j][q] = x[j];
    }
    const int64_t ok = k0 + 16 * kb;
    if (ok < ldbt) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t on = n0 + 4 * w + j;
        if (on < n)
          *reinterpret_cast<uint4*>(Bt + on * ldbt + ok) = make_uint4(o[j][0], o[j][1], o[j][2],
                                                                      o[j][3]);
      }
    }
    __syncthreads();
  }
}

// Asynchronous copies need 16-byte aligned rows.
bool rows_aligned(const void* p, int64_t ld) {
  return ((reinterpret_cast<uintptr_t>(p) & 15) == 0) && ld % 8 == 0;
}

// bf16 elements in a 256-byte aligned plane of `elems` elements.
int64_t align_elems(int64_t elems) { return (elems * 2 + 255) / 256 * 128; }

}  // namespace

// Native FP8 data tiles (the e4m3 codes on the 8-bit tensor path) unless the
// environment variable ABFT_FP8_NATIVE is 0, which multiplies the dequantised
// bf16 planes instead (for comparison; the encode and the product of a
// workspace must see the same setting).
static bool fp8_native() {
  const char* env = getenv("ABFT_FP8_NATIVE");
  return !(env && env[0] == '0');
}

// A byte matrix whose base and row pitch are 16-byte multiples (TMA rows).
static bool aligned16(const void* p, int64_t ld_bytes) {
  return p && ((reinterpret_cast<uintptr_t>(p) & 15) == 0) && ld_bytes % 16 == 0;
}

// Scratch of the tensor-core encode, carved from the workspace's partial-sum
// region: checksum-norm partials (binary64), then per-row and per-column
// partial sums of squares (fp32).
size_t lp_part_bytes(const Plan& P) {
  const int64_t k = P.d.k > 0 ? P.d.k : 1;
  return sizeof(double) * (2 * P.nvr * cdiv(k, kEncCols) + 2 * P.nvc * cdiv(k, kRowsPerCtaB)) +
         sizeof(float) * (P.d.m * cdiv(k, 256) + cdiv(k, kRowsPerCtaB) * P.d.n) + 64;
}

cudaError_t launch_encode_lp(const Plan& P, const void* Av, const void* Bv, const void* a_scale,
                             const void* b_scale, void* ws, cudaStream_t st) {
  const abft_desc& d = P.d;
  const auto* A = static_cast<const __nv_bfloat16*>(Av);
  const auto* B = static_cast<const __nv_bfloat16*>(Bv);
  int64_t lda = d.lda, ldb = d.ldb;
  char* w = static_cast<char*>(ws);
  auto* acs = reinterpret_cast<__nv_bfloat16*>(w + P.L.acs);
  auto* bcs = reinterpret_cast<__nv_bfloat16*>(w + P.L.bcs);
  double* nArow = reinterpret_cast<double*>(w + P.L.nArow);
  double* nAblk = reinterpret_cast<double*>(w + P.L.nAblk);
  double* nBcol = reinterpret_cast<double*>(w + P.L.nBcol);
  double* nBblk = reinterpret_cast<double*>(w + P.L.nBblk);
  Scratch S = scratch_view(P, ws);
  if (d.k == 0) {
    cudaMemsetAsync(nArow, 0, sizeof(double) * d.m, st);
    cudaMemsetAsync(nAblk, 0, sizeof(double) * 4 * P.nvr, st);
    cudaMemsetAsync(nBcol, 0, sizeof(double) * d.n, st);
    cudaMemsetAsync(nBblk, 0, sizeof(double) * 4 * P.nvc, st);
    return cudaGetLastError();
  }
  const int64_t nchA = cdiv(d.k, kColsPerCta);
  const int64_t nchB = cdiv(d.k, kRowsPerCtaB);
  const int64_t nchr = cdiv(d.k, 256);
  double* partA = S.part;
  double* partB = partA + 2 * P.nvr * nchr;  // room for the bf16 pass's ceil(k/256) partials
  float* rowpart = reinterpret_cast<float*>(partB + 2 * P.nvc * nchB);
  float* colpart = rowpart + d.m * nchr;
  const bool fastB = d.vb_cols >= 8 && d.vb_cols <= 256 && (d.vb_cols & (d.vb_cols - 1)) == 0;
  for (int pl = 0; pl < P.L.planes; ++pl)
    if (P.L.bcs_ld > P.L.bcs_cols)
      cudaMemset2DAsync(reinterpret_cast<char*>(bcs) + pl * P.L.bcs_plane + P.L.bcs_cols * 2,
                        P.L.bcs_ld * 2, 0, (P.L.bcs_ld - P.L.bcs_cols) * 2, d.k, st);
  if (d.dtype == ABFT_BF16X3 || d.dtype == ABFT_BF16X6) {
    const float* Af = static_cast<const float*>(Av);
    const float* Bf = static_cast<const float*>(Bv);
    const int np = P.L.planes;
    Planes opa{}, opb{}, acsp{}, bcsp{};
    opa.np = opb.np = acsp.np = bcsp.np = np;
    for (int i = 0; i < np; ++i) {
      opa.p[i] = reinterpret_cast<__nv_bfloat16*>(w + P.L.op_a) + i * align_elems(d.m * P.L.op_a_ld);
      opb.p[i] = reinterpret_cast<__nv_bfloat16*>(w + P.L.op_b) + i * align_elems(d.k * P.L.op_b_ld);
      acsp.p[i] = reinterpret_cast<__nv_bfloat16*>(w + P.L.acs + i * P.L.acs_plane);
      bcsp.p[i] = reinterpret_cast<__nv_bfloat16*>(w + P.L.bcs + i * P.L.bcs_plane);
    }
    k_x3A_cols<<<dim3((unsigned)nchA, gy(P.nvr)), kThreads, 0, st>>>(
        Af, d.lda, d.m, d.k, d.vb_rows, P.er, opa, acsp, P.L.acs_ld, rowpart, nchr, partA, nchA,
        1);
    if (P.bs > 0) {
      Planes sp = acsp;
      for (int i = 0; i < np; ++i) sp.p[i] += 2 * P.nvr * P.L.acs_ld;
      k_x3A_block<<<dim3((unsigned)cdiv(d.k, kThreads), gy(P.f * P.bs)), kThreads, 0, st>>>(
          Af, d.lda, d.k, d.grid_p, P.bs, P.f, sp, P.L.acs_ld);
    }
    k_lp_norms_blk<<<(unsigned)P.nvr, kThreads, 0, st>>>(rowpart, d.m, nchr, nchr, 1, nArow,
                                                       d.vb_rows, P.er, partA, nchA, nAblk);
    if (fastB) {
      k_x3B_rows<<<dim3((unsigned)cdiv(P.L.op_b_ld, kColsPerCta), (unsigned)nchB), kThreads, 0,
                   st>>>(
          Bf, d.ldb, d.k, d.n, d.vb_cols, P.ec, opb, P.L.op_b_ld, bcsp, P.L.bcs_ld, colpart,
          partB, nchB);
    } else {
      k_x3B_split<<<dim3((unsigned)cdiv(P.L.op_b_ld, kThreads), gy(nchB)), kThreads, 0, st>>>(
          Bf, d.ldb, d.k, d.n, opb, P.L.op_b_ld, colpart);
      k_x3B_rows_any<<<dim3((unsigned)cdiv(nchB, kThreads / 32), gy(P.nvc)), kThreads, 0, st>>>(
          Bf, d.ldb, d.k, d.n, d.vb_cols, P.ec, bcsp, P.L.bcs_ld, partB, nchB);
    }
    k_lp_norms_blk<<<(unsigned)P.nvc, kThreads, 0, st>>>(colpart, d.n, nchB, 1, d.n, nBcol,
                                                       d.vb_cols, P.ec, partB, nchB, nBblk);
    count_launches(4 + (P.bs > 0 ? 1 : 0) + (fastB ? 0 : 1));
    return cudaGetLastError();
  }
  // FP8: the exact dequantised values go to bf16 operand planes, which the
  // checksums and the product use.  With 8-byte aligned e4m3 rows the
  // streaming passes dequantise as they read (one pass over each operand);
  // otherwise a dequantisation pass writes the planes first.
  bool f8A = false, f8B = false;
  Fp8Src fa{}, fb{};
  int nlaunch = 0;
  if (d.dtype == ABFT_FP8_E4M3) {
    // this workspace's status word of its last encode (read by the verify)
    int* flag = S.cnt + kCntFp8Inexact;
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    // the block scales, for the product's native FP8 data tiles
    const size_t nsa = (size_t)(cdiv(d.m, 128) * cdiv(d.k, 128));
    const size_t nsb = (size_t)(cdiv(d.k, 128) * cdiv(d.n, 128));
    e = cudaMemcpyAsync(w + P.L.scales, a_scale, sizeof(float) * nsa, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(w + P.L.scales + sizeof(float) * nsa, b_scale, sizeof(float) * nsb,
                          cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    auto* pa = reinterpret_cast<__nv_bfloat16*>(w + P.L.op_a);
    auto* pb = reinterpret_cast<__nv_bfloat16*>(w + P.L.op_b);
    const auto* qa = static_cast<const uint8_t*>(Av);
    const auto* qb = static_cast<const uint8_t*>(Bv);
    fa = Fp8Src{qa, d.lda, static_cast<const float*>(a_scale), cdiv(d.k, 128), pa, P.L.op_a_ld,
                flag, nullptr, 0};
    fb = Fp8Src{qb, d.ldb, static_cast<const float*>(b_scale), cdiv(d.n, 128), pb, P.L.op_b_ld,
                flag, nullptr, 0};
    f8A = ((reinterpret_cast<uintptr_t>(qa) & 7) == 0) && d.lda % 8 == 0;
    f8B = ((reinterpret_cast<uintptr_t>(qb) & 7) == 0) && d.ldb % 8 == 0 && fastB;
    // B^T of the codes and the scale groups of the data tiles, for the
    // product's native data tiles (K-major B); the streaming B pass writes
    // B^T as it reads B, else a transposing pass does
    if (fp8_native() && aligned16(Av, d.lda) && aligned16(Bv, d.ldb)) {
      const float* ws_sa = reinterpret_cast<const float*>(w + P.L.scales);
      e = launch_f8_groups(ws_sa, ws_sa + nsa, d.m, d.n, d.k,
                           reinterpret_cast<uint32_t*>(w + P.L.f8grp), st);
      if (e != cudaSuccess) return e;
      const int64_t ldbt = (d.k + 15) / 16 * 16;
      if (f8B) {
        fb.bt = reinterpret_cast<uint8_t*>(w + P.L.f8bt);
        fb.ldbt = ldbt;
      } else {
        k_transpose_u8<<<dim3((unsigned)cdiv(d.n, 128), gy(cdiv(ldbt, 128))), 256, 0, st>>>(
            qb, d.ldb, d.k, d.n, reinterpret_cast<uint8_t*>(w + P.L.f8bt), ldbt);
        ++nlaunch;
      }
    }
    if (!f8A) {
      k_fp8_dequant<<<dim3((unsigned)cdiv(P.L.op_a_ld, 8 * kThreads), gy(cdiv(d.m, kDqRows))),
                      kThreads, 0, st>>>(qa, d.lda, d.m, d.k, fa.sc, pa, P.L.op_a_ld, flag);
      ++nlaunch;
    }
    if (!f8B) {
      k_fp8_dequant<<<dim3((unsigned)cdiv(P.L.op_b_ld, 8 * kThreads), gy(cdiv(d.k, kDqRows))),
                      kThreads, 0, st>>>(qb, d.ldb, d.k, d.n, fb.sc, pb, P.L.op_b_ld, flag);
      ++nlaunch;
    }
    A = pa;
    B = pb;
    lda = P.L.op_a_ld;
    ldb = P.L.op_b_ld;
  }
  if (f8A || rows_aligned(A, lda)) {
    SingleAUnits U{};
    U.base = EncAUnit{A, lda, d.m, d.k, d.vb_rows, P.er, acs, P.L.acs_ld, rowpart, nchr, partA, 0, 0};
    U.ncx = cdiv(P.L.acs_ld, kEncCols);
    U.cnt = U.ncx * P.nvr;
    cudaError_t e = f8A ? launch_stream_A<SingleAUnits, true>(U, st, fa) : launch_stream_A(U, st);
    if (e != cudaSuccess) return e;
  } else {
    k_lpA_cols<<<dim3((unsigned)cdiv(P.L.acs_ld, kEncCols), gy(P.nvr)), kThreads, 0, st>>>(
        A, lda, d.m, d.k, d.vb_rows, P.er, acs, P.L.acs_ld, rowpart, nchr, partA);
    ++nlaunch;
  }
  if (P.bs > 0)
    k_lpA_block<<<dim3((unsigned)cdiv(d.k, kThreads), gy(P.f * P.bs)), kThreads, 0, st>>>(
        A, lda, d.k, d.grid_p, P.bs, P.f, acs + 4 * P.nvr * P.L.acs_ld, P.L.acs_ld);
  k_lp_norms_blk<<<(unsigned)P.nvr, kThreads, 0, st>>>(rowpart, d.m, nchr, nchr, 1, nArow,
                                                     d.vb_rows, P.er, partA, nchr, nAblk);
  if (f8B || (fastB && rows_aligned(B, ldb))) {
    SingleBUnits U{};
    U.base = EncBUnit{B, ldb, d.k, d.n, d.vb_cols, P.ec, bcs, P.L.bcs_ld, colpart, partB, nchB,
                      0, 0};
    U.ncx = cdiv(d.n, kEncCols);
    U.cnt = U.ncx * nchB;
    cudaError_t e = f8B ? launch_stream_B<SingleBUnits, true>(U, st, fb) : launch_stream_B(U, st);
    if (e != cudaSuccess) return e;
  } else if (fastB) {
    k_lpB_rows<<<dim3((unsigned)cdiv(d.n, kEncCols), gy(nchB)), kThreads, 0, st>>>(
        B, ldb, d.k, d.n, d.vb_cols, P.ec, bcs, P.L.bcs_ld, colpart, partB, nchB);
    ++nlaunch;
  } else {
    k_lpB_rows_any<<<dim3((unsigned)cdiv(nchB, kThreads / 32), gy(P.nvc)), kThreads, 0, st>>>(
        B, ldb, d.k, d.n, d.vb_cols, P.ec, bcs, P.L.bcs_ld, partB, nchB);
    k_lp_col_sq<<<dim3((unsigned)cdiv(d.n, kThreads), gy(nchB)), kThreads, 0, st>>>(
        B, ldb, d.k, d.n, colpart);
  }
  k_lp_norms_blk<<<(unsigned)P.nvc, kThreads, 0, st>>>(colpart, d.n, nchB, 1, d.n, nBcol,
                                                     d.vb_cols, P.ec, partB, nchB, nBblk);
  count_launches(nlaunch + 2 + (P.bs > 0 ? 1 : 0) + (fastB ? 0 : 2));
  return cudaGetLastError();
}

cudaError_t launch_encode_lp_chained(const Plan& P, const void* Av, const void* Bv, void* ws,
                                     const Plan* PL, const void* wsL, const Plan* PR,
                                     const void* wsR, cudaStream_t st) {
  const abft_desc& d = P.d;
  if (d.k == 0 || (!PL && !PR)) return launch_encode_lp(P, Av, Bv, nullptr, nullptr, ws, st);
  char* w = static_cast<char*>(ws);
  double* nArow = reinterpret_cast<double*>(w + P.L.nArow);
  double* nAblk = reinterpret_cast<double*>(w + P.L.nAblk);
  double* nBcol = reinterpret_cast<double*>(w + P.L.nBcol);
  double* nBblk = reinterpret_cast<double*>(w + P.L.nBblk);
  double* carA = reinterpret_cast<double*>(w + P.L.car_a);
  double* carB = reinterpret_cast<double*>(w + P.L.car_b);
  Scratch S = scratch_view(P, ws);
  const int64_t nchA = cdiv(d.k, kColsPerCta);
  const int64_t nchB = cdiv(d.k, kRowsPerCtaB);
  const int64_t nchr = cdiv(d.k, 256);
  double* partA = S.part;
  double* partB = partA + 2 * P.nvr * nchr;
  float* rowpart = reinterpret_cast<float*>(partB + 2 * P.nvc * nchB);
  float* colpart = rowpart + d.m * nchr;
  const bool fastB = d.vb_cols >= 8 && d.vb_cols <= 256 && (d.vb_cols & (d.vb_cols - 1)) == 0;
  const float* Af = static_cast<const float*>(Av);
  const float* Bf = static_cast<const float*>(Bv);
  const int np = P.L.planes;
  Planes opa{}, opb{}, acsp{}, bcsp{};
  opa.np = opb.np = acsp.np = bcsp.np = np;
  for (int i = 0; i < np; ++i) {
    opa.p[i] = reinterpret_cast<__nv_bfloat16*>(w + P.L.op_a) + i * align_elems(d.m * P.L.op_a_ld);
    opb.p[i] = reinterpret_cast<__nv_bfloat16*>(w + P.L.op_b) + i * align_elems(d.k * P.L.op_b_ld);
    acsp.p[i] = reinterpret_cast<__nv_bfloat16*>(w + P.L.acs + i * P.L.acs_plane);
    bcsp.p[i] = reinterpret_cast<__nv_bfloat16*>(w + P.L.bcs + i * P.L.bcs_plane);
  }
  for (int pl = 0; pl < np; ++pl)
    if (P.L.bcs_ld > P.L.bcs_cols)
      cudaMemset2DAsync(reinterpret_cast<char*>(bcsp.p[pl]) + P.L.bcs_cols * 2, P.L.bcs_ld * 2, 0,
                        (P.L.bcs_ld - P.L.bcs_cols) * 2, d.k, st);
  int launches = 0;
  cudaError_t e = cudaSuccess;
  // A: operand planes and row norms from A; checksum rows carried (E of the
  // earlier product: verify rows, then block checksum rows) or formed
  k_x3A_cols<<<dim3((unsigned)nchA, gy(P.nvr)), kThreads, 0, st>>>(
      Af, d.lda, d.m, d.k, d.vb_rows, P.er, opa, acsp, P.L.acs_ld, rowpart, nchr, partA, nchA,
      PL ? 0 : 1);
  ++launches;
  if (PL) {
    const double* EL = reinterpret_cast<const double*>(static_cast<const char*>(wsL) + PL->L.E);
    k_carried_rows_split<<<dim3((unsigned)nchA, gy(P.R)), kThreads, 0, st>>>(
        EL, P.R, d.k, acsp, P.L.acs_ld, partA, nchA, 2 * P.nvr);
    if ((e = launch_carry_rows(*PL, wsL, carA, st)) != cudaSuccess) return e;
    launches += 2;
  } else if (P.bs > 0) {
    Planes sp = acsp;
    for (int i = 0; i < np; ++i) sp.p[i] += 2 * P.nvr * P.L.acs_ld;
    k_x3A_block<<<dim3((unsigned)cdiv(d.k, kThreads), gy(P.f * P.bs)), kThreads, 0, st>>>(
        Af, d.lda, d.k, d.grid_p, P.bs, P.f, sp, P.L.acs_ld);
    ++launches;
  }
  k_lp_norms_blk<<<(unsigned)P.nvr, kThreads, 0, st>>>(rowpart, d.m, nchr, nchr, 1, nArow,
                                                     d.vb_rows, P.er, partA, nchA, nAblk);
  ++launches;
  // B: operand planes and column norms from B; checksum columns carried (F of
  // the earlier product) or formed
  if (PR) {
    k_x3B_split<<<dim3((unsigned)cdiv(P.L.op_b_ld, kThreads), gy(nchB)), kThreads, 0, st>>>(
        Bf, d.ldb, d.k, d.n, opb, P.L.op_b_ld, colpart);
    const double* FR = reinterpret_cast<const double*>(static_cast<const char*>(wsR) + PR->L.F);
    k_carried_cols_split<<<(unsigned)cdiv(P.Cc * nchB, kThreads), kThreads, 0, st>>>(
        FR, d.k, P.Cc, bcsp, P.L.bcs_ld, partB, nchB);
    if ((e = launch_carry_cols(*PR, wsR, carB, st)) != cudaSuccess) return e;
    launches += 3;
  } else if (fastB) {
    k_x3B_rows<<<dim3((unsigned)cdiv(P.L.op_b_ld, kColsPerCta), (unsigned)nchB), kThreads, 0,
                 st>>>(Bf, d.ldb, d.k, d.n, d.vb_cols, P.ec, opb, P.L.op_b_ld, bcsp, P.L.bcs_ld,
                       colpart, partB, nchB);
    ++launches;
  } else {
    k_x3B_split<<<dim3((unsigned)cdiv(P.L.op_b_ld, kThreads), gy(nchB)), kThreads, 0, st>>>(
        Bf, d.ldb, d.k, d.n, opb, P.L.op_b_ld, colpart);
    k_x3B_rows_any<<<dim3((unsigned)cdiv(nchB, kThreads / 32), gy(P.nvc)), kThreads, 0, st>>>(
        Bf, d.ldb, d.k, d.n, d.vb_cols, P.ec, bcsp, P.L.bcs_ld, partB, nchB);
    launches += 2;
  }
  k_lp_norms_blk<<<(unsigned)P.nvc, kThreads, 0, st>>>(colpart, d.n, nchB, 1, d.n, nBcol,
                                                     d.vb_cols, P.ec, partB, nchB, nBblk);
  ++launches;
  count_launches(launches);
  return cudaGetLastError();
}

cudaError_t launch_gemm_lp(const Plan& P, const void* A, const void* B, float* C, void* ws,
                           bool checksums, cudaStream_t st) {
  const abft_desc& d = P.d;
  char* w = static_cast<char*>(ws);
  if (d.k == 0) {  // empty inner dimension: every product is zero
    cudaError_t e = cudaMemset2DAsync(C, d.ldc * 4, 0, d.n * 4, d.m, st);
    if (e == cudaSuccess && checksums) {
      e = cudaMemsetAsync(w + P.L.E, 0, (size_t)P.R * d.n * 8, st);
      if (e == cudaSuccess) e = cudaMemsetAsync(w + P.L.F, 0, (size_t)d.m * P.Cc * 8, st);
    }
    return e;
  }
  TcOperands op{};
  if (d.dtype == ABFT_BF16X3 || d.dtype == ABFT_BF16X6) {
    const auto* pa = reinterpret_cast<const __nv_bfloat16*>(w + P.L.op_a);
    const auto* pb = reinterpret_cast<const __nv_bfloat16*>(w + P.L.op_b);
    for (int i = 0; i < 3; ++i) {
      const int pl = i < P.L.planes ? i : 0;
      op.a[i] = pa + pl * align_elems(d.m * P.L.op_a_ld);
      op.b[i] = pb + pl * align_elems(d.k * P.L.op_b_ld);
    }
    op.lda = P.L.op_a_ld;
    op.ldb = P.L.op_b_ld;
    if (d.dtype == ABFT_BF16X3) {
      // A0 B0, A0 B1, A1 B0
      op.nseg = 3;
      op.seg_a = 0u | (0u << 2) | (1u << 4);
      op.seg_b = 0u | (1u << 2) | (0u << 4);
    } else {
      // the six products with a + b <= 2, smallest first: A2 B0, A1 B1, A0 B2,
      // A1 B0, A0 B1, A0 B0
      op.nseg = 6;
      op.seg_a = 2u | (1u << 2) | (0u << 4) | (1u << 6) | (0u << 8) | (0u << 10);
      op.seg_b = 0u | (1u << 2) | (2u << 4) | (0u << 6) | (1u << 8) | (0u << 10);
    }
  } else if (d.dtype == ABFT_FP8_E4M3) {
    // checksum tiles: the exact dequantised bf16 planes abft_encode wrote; data
    // tiles: the e4m3 codes on the 8-bit tensor path when their rows suit TMA
    // (16-byte aligned), else the planes too
    op.a[0] = op.a[1] = op.a[2] = w + P.L.op_a;
    op.b[0] = op.b[1] = op.b[2] = w + P.L.op_b;
    op.lda = P.L.op_a_ld;
    op.ldb = P.L.op_b_ld;
    op.nseg = 1;
    if (fp8_native() && aligned16(A, d.lda) && aligned16(B, d.ldb)) {
      op.a8 = A;
      op.b8 = w + P.L.f8bt;  // B^T, written by the encode
      op.lda8 = d.lda;
      op.ldb8 = (d.k + 15) / 16 * 16;
      op.sA = reinterpret_cast<const float*>(w + P.L.scales);
      op.sB = op.sA + cdiv(d.m, 128) * cdiv(d.k, 128);
      op.f8grp = reinterpret_cast<uint32_t*>(w + P.L.f8grp);
    }
  } else {
    op.a[0] = op.a[1] = op.a[2] = A;
    op.b[0] = op.b[1] = op.b[2] = B;
    op.lda = d.lda;
    op.ldb = d.ldb;
    op.nseg = 1;
  }
  // a timeout goes to this workspace's status word (read by the verify); a
  // checksum-free product without a workspace has no report to carry it
  int* status = nullptr;
  cudaError_t e = ws ? cudaSuccess : tc_timeout_fallback(&status);
  if (e != cudaSuccess) return e;
  if (ws) status = scratch_view(P, ws).cnt + kCntTimeout;
  e = launch_gemm_bf16(P, op, C, ws, checksums, status, st);
  if (e != cudaSuccess || !checksums) return e;
  const int npc = (d.dtype == ABFT_BF16X3 || d.dtype == ABFT_BF16X6) ? 1 : 2;
  const float* E16 = reinterpret_cast<const float*>(w + P.L.E16);
  const float* F16 = reinterpret_cast<const float*>(w + P.L.F16);
  double* E = reinterpret_cast<double*>(w + P.L.E);
  double* F = reinterpret_cast<double*>(w + P.L.F);
  k_fold_E<<<dim3((unsigned)cdiv(d.n, 256), gy(P.R)), 256, 0, st>>>(E16, P.R, npc, d.n, E);
  k_fold_F<<<(unsigned)cdiv(d.m * P.Cc, 256), 256, 0, st>>>(F16, d.m, P.Cc, P.L.bcs_cols, npc, F);
  count_launches(2);
  return cudaGetLastError();
}

// ---------------- grouped encode (many bf16 problems per launch)
namespace {

// Row norms ||A_i|| (first ceil(m/256) CTAs of a problem) and column norms
// ||B_:j|| (next ceil(n/256)) from the fp32 partial sums of squares (fp32
// sums; stored as binary64 and as fp32 for the verify screen).
__global__ void __launch_bounds__(kThreads) k_grp_lines(const GProb* __restrict__ probs,
                                                        const int2* __restrict__ tab) {
  const int2 e = tab[blockIdx.x];
  const GProb& P = probs[e.x];
  const int64_t u = e.y, nra = cdiv(P.m, kThreads);
  if (u < nra) {
    const int64_t i = u * kThreads + threadIdx.x;
    if (i >= P.m) return;
    const int64_t nchr = cdiv(P.k, 256);
    float s = 0.f;
    for (int64_t c = 0; c < nchr; ++c) s += P.rowpart[i * nchr + c];
    s = sqrtf(s);
    P.nArow[i] = (double)s;
    P.nArow32[i] = s;
  } else {
    const int64_t j = (u - nra) * kThreads + threadIdx.x;
    if (j >= P.n) return;
    const int64_t nch = cdiv(P.k, kRowsPerCtaB);
    float s = 0.f;
    for (int64_t c = 0; c < nch; ++c) s += P.colpart[c * P.n + j];
    s = sqrtf(s);
    P.nBcol[j] = (double)s;
    P.nBcol32[j] = s;
  }
}

// Threshold norms of every verify block and the fp32 threshold factors of
// the verify screen; one CTA per problem.
// The threshold norms of verify block I (as k_lp_norms_blk forms them, from
// line norms already stored) with one warp: lanes over the block's lines and
// partials, fp32 sums combined by shuffles, lane 0 stores.
__device__ __forceinline__ void lp_blk_warp(const double* __restrict__ nvec, int64_t len, int vb,
                                            int e, const double* __restrict__ part, int64_t nch,
                                            double* __restrict__ nblk, int64_t I, int lane) {
  const float sc = scalbnf(1.0f, -e);
  const int64_t t0 = I * vb, t1 = min(t0 + (int64_t)vb, len);
  float f0 = 0.f, f1 = 0.f, q0 = 0.f, q1 = 0.f;
  for (int64_t t = t0 + lane; t < t1; t += 32) {
    const float v = (float)nvec[t], wv = (float)(t - t0 + 1) * sc * v;
    f0 = fmaf(v, v, f0);
    f1 = fmaf(wv, wv, f1);
  }
  for (int64_t c = lane; c < nch; c += 32) {
    q0 += (float)part[(2 * I) * nch + c];
    q1 += (float)part[(2 * I + 1) * nch + c];
  }
  f0 = warp_sumf(f0);
  f1 = warp_sumf(f1);
  q0 = warp_sumf(q0);
  q1 = warp_sumf(q1);
  if (lane == 0) {
    nblk[4 * I + 0] = (double)sqrtf(f0);
    nblk[4 * I + 1] = (double)sqrtf(f1);
    nblk[4 * I + 2] = (double)sqrtf(q0);
    nblk[4 * I + 3] = (double)sqrtf(q1);
  }
}

// The verify blocks' threshold norms and fp32 thresholds of one problem per
// CTA: one warp per verify block (row blocks of A, then column blocks of B).
__global__ void __launch_bounds__(kThreads) k_grp_blk(const GProb* __restrict__ probs, double s) {
  const GProb& P = probs[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t t = warp; t < P.nvr + P.nvc; t += kThreads / 32) {
    if (t < P.nvr) {
      lp_blk_warp(P.nArow, P.m, kGrpVbR, kGrpEr, P.partA, cdiv(P.k, kEncCols), P.nAblk, t, lane);
      if (lane == 0) {
        const double* nb = P.nAblk + 4 * t;
        P.tauA[2 * t + 0] = (float)(s * (P.f1c * nb[0] + P.f2 * nb[2]));
        P.tauA[2 * t + 1] = (float)(s * (P.f1c * nb[1] + P.f2 * nb[3]));
      }
    } else {
      const int64_t J = t - P.nvr;
      lp_blk_warp(P.nBcol, P.n, kGrpVbC, kGrpEc, P.partB, cdiv(P.k, kRowsPerCtaB), P.nBblk, J,
                  lane);
      if (lane == 0) {
        const double* nb = P.nBblk + 4 * J;
        P.tauB[2 * J + 0] = (float)(s * (P.f1r * nb[0] + P.f2 * nb[2]));
        P.tauB[2 * J + 1] = (float)(s * (P.f1r * nb[1] + P.f2 * nb[3]));
      }
    }
  }
}

}  // namespace

cudaError_t launch_group_encode(const GroupDev& G, cudaStream_t st) {
  if (G.count == 0) return cudaSuccess;
  // (every problem's operands have 16-byte aligned rows: their tensor maps need it)
  cudaError_t e = launch_stream_A(GroupAUnits{G.probs, G.tab[kGkEncA], G.nctas[kGkEncA]}, st);
  if (e == cudaSuccess)
    e = launch_stream_B(GroupBUnits{G.probs, G.tab[kGkEncB], G.nctas[kGkEncB]}, st);
  if (e != cudaSuccess) return e;
  if (G.nctas[kGkLines] > 0)
    k_grp_lines<<<(unsigned)G.nctas[kGkLines], kThreads, 0, st>>>(G.probs, G.tab[kGkLines]);
  k_grp_blk<<<(unsigned)G.count, kThreads, 0, st>>>(G.probs, G.s);
  count_launches(2);
  return cudaGetLastError();
}

}  // namespace abft
