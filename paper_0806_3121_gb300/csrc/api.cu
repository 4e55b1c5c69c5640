// Host side of the C ABI declared in include/abft.h: descriptor validation,
// workspace layout, launches, report collection.  No exception crosses the
// ABI; failures return a status and set a thread-local message.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "internal.cuh"

namespace abft {

thread_local char g_err[512] = "";

abft_status fail(abft_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return st;
}

// Workspaces must be 256-byte aligned (every region offset is a multiple of
// 256 from the base: TMA maps, vector loads and stores rely on it).
bool ws_misaligned(const void* ws) { return (reinterpret_cast<uintptr_t>(ws) & 255) != 0; }

abft_status cuda_fail(cudaError_t e, const char* where) {
  return fail(ABFT_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

namespace {

std::atomic<int64_t> g_launches{0};

int ceil_log2(int64_t v) {
  int e = 0;
  while (((int64_t)1 << e) < v) ++e;
  return e;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Unit roundoffs entering the detection threshold:
//   u_acc: accumulation of the product, u_sum: observed block sums,
//   u_enc: checksum encoding sums, u_c: storage rounding of C relative to
//   the accumulator, u_cs: representation error of the checksum operand.
struct Units {
  double u_acc, u_sum, u_enc, u_c, u_cs;
};
Units units_for(int dtype) {
  const double u64 = ldexp(1.0, -53), u32 = ldexp(1.0, -24);
  if (dtype == ABFT_F64) return {u64, u64, u64, u64, u64};
  // BF16X3: C also differs from the exact product of the fp32 inputs by the
  // dropped A_lo B_lo term and the hi+lo representation (2^-17 relative).
  if (dtype == ABFT_BF16X3) return {u32, u32, u32, ldexp(1.0, -17), ldexp(1.0, -17)};
  // BF16X6: three pieces keep 24 bits; the dropped products and the pieces'
  // residual stay below 2^-25 of a product, 2^-26 of a checksum.
  if (dtype == ABFT_BF16X6) return {u32, u32, u32, ldexp(1.0, -25), ldexp(1.0, -26)};
  return {u32, u32, u32, 0.0, ldexp(1.0, -17)};
}

}  // namespace

void threshold_factors(int dtype, int64_t k, int64_t vb_r, int64_t vb_c, double* f1_col,
                       double* f1_row, double* f2) {
  const Units u = units_for(dtype);
  const double sk = sqrt((double)k);
  *f1_col = sk * u.u_acc + sqrt((double)vb_r) * (u.u_sum + u.u_enc) + u.u_c;
  *f1_row = sk * u.u_acc + sqrt((double)vb_c) * (u.u_sum + u.u_enc) + u.u_c;
  *f2 = sk * u.u_acc + u.u_cs;
}

namespace {

size_t operand_bytes(int dtype) { return dtype == ABFT_F64 ? 8 : 2; }  // of acs / bcs

abft_status make_plan(const abft_desc* d, Plan* P) {
  if (!d) return fail(ABFT_ERR_INVALID, "desc is NULL");
  if (d->dtype != ABFT_F64 && d->dtype != ABFT_BF16 && d->dtype != ABFT_BF16X3 &&
      d->dtype != ABFT_FP8_E4M3 && d->dtype != ABFT_BF16X6)
    return fail(ABFT_ERR_INVALID, "unknown dtype %d", d->dtype);
  if (d->m < 0 || d->n < 0 || d->k < 0) return fail(ABFT_ERR_INVALID, "negative size");
  if (d->m > (1ll << 22) || d->n > (1ll << 22) || d->k >= (1ll << 31))
    return fail(ABFT_ERR_INVALID, "m, n must be at most 2^22 and k below 2^31");
  if (d->lda < std::max<int64_t>(d->k, 1) || d->ldb < std::max<int64_t>(d->n, 1) ||
      d->ldc < std::max<int64_t>(d->n, 1))
    return fail(ABFT_ERR_INVALID, "leading dimension too small (lda>=k, ldb>=n, ldc>=n)");
  if (d->vb_rows < 1 || d->vb_cols < 1 || (d->m > 0 && d->vb_rows > d->m) ||
      (d->n > 0 && d->vb_cols > d->n))
    return fail(ABFT_ERR_INVALID, "verify block sizes must be in [1, m] x [1, n]");
  if (d->grid_p < 0 || d->grid_q < 0 || (d->grid_p > 0) != (d->grid_q > 0))
    return fail(ABFT_ERR_INVALID, "erasure grid: grid_p and grid_q both 0 or both > 0");
  if (d->grid_p > 0 && (d->m % d->grid_p || d->n % d->grid_q))
    return fail(ABFT_ERR_INVALID, "erasure grid must divide m and n");
  if (d->flags != 0 || d->reserved != 0) return fail(ABFT_ERR_INVALID, "flags must be 0");
  if (d->grid_f < 0 || d->grid_f > kMaxBlockChecksums)
    return fail(ABFT_ERR_INVALID, "grid_f must be in [0, %d]", kMaxBlockChecksums);
  if (d->grid_p > 0 && d->grid_f > d->grid_p)
    return fail(ABFT_ERR_INVALID, "grid_f larger than the number of block rows");
  if (!(d->tau_safety >= 0.0) || !isfinite(d->tau_safety))
    return fail(ABFT_ERR_INVALID, "tau_safety must be finite and >= 0");

  if (d->dtype == ABFT_BF16 && (d->lda % 8 || d->ldb % 8))  // TMA rows of A and B
    return fail(ABFT_ERR_INVALID, "bf16 operands need lda and ldb multiples of 8 (16-byte rows)");

  Plan& p = *P;
  memset(&p, 0, sizeof p);
  p.d = *d;
  p.nvr = d->m > 0 ? cdiv(d->m, d->vb_rows) : 0;
  p.nvc = d->n > 0 ? cdiv(d->n, d->vb_cols) : 0;
  p.bs = d->grid_p > 0 ? d->m / d->grid_p : 0;
  p.bc = d->grid_q > 0 ? d->n / d->grid_q : 0;
  p.f = d->grid_f > 0 ? d->grid_f : 1;
  p.R = 2 * p.nvr + p.f * p.bs;
  p.Cc = 2 * p.nvc;
  p.er = ceil_log2(d->vb_rows);
  p.ec = ceil_log2(d->vb_cols);
  p.s = d->tau_safety > 0 ? d->tau_safety : 4.0;
  threshold_factors(d->dtype, d->k, d->vb_rows, d->vb_cols, &p.f1_col, &p.f1_row, &p.f2_col);
  p.f2_row = p.f2_col;
  const bool lp0 = d->dtype != ABFT_F64;
  p.fused = lp0 && d->vb_rows % 128 == 0 && d->vb_cols % 32 == 0 &&
            (256 % d->vb_cols == 0 || d->vb_cols % 256 == 0);
  p.g = d->vb_cols < 128 ? d->vb_cols : 128;  // row-sum groups never straddle 128 columns
  p.ngrp = d->n > 0 ? cdiv(d->n, p.g) : 0;
  p.ntr_obs = d->m > 0 ? cdiv(d->m, 32) : 0;  // observed column sums per 32 rows


  abft_ws_layout& L = p.L;
  const size_t eb = operand_bytes(d->dtype);
  const bool lp = d->dtype != ABFT_F64;
  const bool x3 = d->dtype == ABFT_BF16X3 || d->dtype == ABFT_BF16X6;  // split binary32 inputs
  const int nsplit = d->dtype == ABFT_BF16X6 ? 3 : 2;
  const bool f8 = d->dtype == ABFT_FP8_E4M3;
  const int op_planes = x3 ? nsplit : (f8 ? 1 : 0);  // bf16 operand planes the encode writes
  // Encoded operand rows/columns: binary64 checksums for F64.  bf16: each fp32
  // checksum is a bf16 hi+lo pair, as separate rows (4 rows per verify block, 2
  // per block-checksum row).  BF16X3: hi and lo planes of 2 rows per block
  // (the split product combines them).  Rows are 16-byte aligned.
  L.planes = x3 ? nsplit : 1;
  L.acs_rows = x3 ? p.R : (lp ? 4 * p.nvr + 2 * p.f * p.bs : p.R);
  L.bcs_cols = x3 ? p.Cc : (lp ? 4 * p.nvc : p.Cc);
  L.acs_ld = lp ? (d->k + 7) / 8 * 8 : d->k;
  L.bcs_ld = lp ? (L.bcs_cols + 7) / 8 * 8 : p.Cc;
  L.acs_plane = align256((size_t)L.acs_rows * L.acs_ld * eb);
  L.bcs_plane = align256((size_t)d->k * L.bcs_ld * eb);
  size_t off = 0;
  auto region = [&](size_t bytes) {
    const size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  L.acs = region(L.acs_plane * L.planes);
  L.bcs = region(L.bcs_plane * L.planes);
  L.E = region((size_t)p.R * d->n * 8);
  L.F = region((size_t)d->m * p.Cc * 8);
  L.nArow = region((size_t)d->m * 8);
  L.nAblk = region((size_t)4 * p.nvr * 8);
  L.nBcol = region((size_t)d->n * 8);
  L.nBblk = region((size_t)4 * p.nvc * 8);
  L.car_a = region((size_t)2 * p.nvr * 8);
  L.car_b = region((size_t)2 * p.nvc * 8);
  L.E16 = region(lp ? (size_t)L.acs_rows * d->n * 4 : 0);
  L.F16 = region(lp ? (size_t)d->m * L.bcs_cols * 4 : 0);
  L.obs_col = region(p.fused ? (size_t)p.ntr_obs * 2 * d->n * 4 : 0);
  L.obs_row = region(p.fused ? (size_t)d->m * p.ngrp * 2 * 4 : 0);
  L.inject = region(lp ? 16 + sizeof(InjectEntry) * kMaxInject : 0);
  L.op_a_ld = op_planes ? (d->k + 7) / 8 * 8 : 0;
  L.op_b_ld = op_planes ? (d->n + 7) / 8 * 8 : 0;
  L.op_a = region(op_planes * align256((size_t)d->m * L.op_a_ld * 2));
  L.op_b = region(op_planes * align256((size_t)d->k * L.op_b_ld * 2));
  // FP8: a copy of the block scales (the product's data tiles scale their e4m3
  // partials by them)
  L.scales = region(f8 ? sizeof(float) * (size_t)(cdiv(d->m, 128) * cdiv(d->k, 128) +
                                                   cdiv(d->k, 128) * cdiv(d->n, 128))
                       : 0);
  // FP8: the transposed copy B^T of the e4m3 codes (n x ceil16(k) bytes), the
  // K-major B operand of the native data tiles
  L.f8bt = region(f8 ? (size_t)d->n * (size_t)((d->k + 15) / 16 * 16) : 0);
  // FP8: per data tile (128 x 256) one bit per 128-wide k-step, set where the
  // block-scale product changes (the product's scale groups)
  L.f8grp = region(f8 ? sizeof(uint32_t) * (size_t)(cdiv(d->m, 128) * cdiv(d->n, 256) *
                                                     cdiv(cdiv(d->k, 128), 32))
                      : 0);
  L.fused = p.fused;
  L.scratch = off;
  L.scratch_bytes = scratch_bytes(p);
  off = align256(off + L.scratch_bytes);
  L.total = off;
  L.R = p.R;
  L.Cc = p.Cc;
  L.nvr = p.nvr;
  L.nvc = p.nvc;
  L.bs = p.bs;
  return ABFT_OK;
}

bool is_empty(const Plan& P) { return P.d.m == 0 || P.d.n == 0; }

// A freshly encoded product carries no checksum deviation, and (tensor-core
// dtypes) its workspace's status words start clear: no product has timed out
// on it and no operand has been found inexact.
cudaError_t clear_carry(const Plan& P, void* ws, cudaStream_t st) {
  char* w = static_cast<char*>(ws);
  cudaError_t e = cudaMemsetAsync(w + P.L.car_a, 0, sizeof(double) * 2 * P.nvr, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(w + P.L.car_b, 0, sizeof(double) * 2 * P.nvc, st);
  if (e == cudaSuccess && P.d.dtype != ABFT_F64)
    e = cudaMemsetAsync(w + P.L.scratch + sizeof(int32_t) * kCntTimeout, 0,
                        sizeof(int32_t) * (kCntFp8Inexact - kCntTimeout + 1), st);
  return e;
}

// Partial-reduction sizes used by the encode kernels (in doubles).
size_t part_elems(const Plan& P) {
  const int64_t k = std::max<int64_t>(P.d.k, 1);
  if (P.d.dtype != ABFT_F64) return (lp_part_bytes(P) + 7) / 8;
  return (size_t)(4 * P.nvr * cdiv(k, 256) + 4 * P.nvc * cdiv(k, 64) + cdiv(k, 256) * P.d.n);
}

}  // namespace

void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

size_t scratch_bytes(const Plan& P) {
  size_t b = 256;  // counters
  b += align256(sizeof(FlagEntry) * kCapFlags) * 2;
  b += align256(sizeof(CandEntry) * kCapCands);
  b += align256(sizeof(abft_fault) * kCapReport);
  b += align256(sizeof(double) * part_elems(P));
  return b;
}

Scratch scratch_view(const Plan& P, void* ws) {
  char* base = static_cast<char*>(ws) + P.L.scratch;
  Scratch S;
  size_t o = 0;
  S.cnt = reinterpret_cast<int32_t*>(base + o);
  o += 256;
  S.colf = reinterpret_cast<FlagEntry*>(base + o);
  o += align256(sizeof(FlagEntry) * kCapFlags);
  S.rowf = reinterpret_cast<FlagEntry*>(base + o);
  o += align256(sizeof(FlagEntry) * kCapFlags);
  S.cand = reinterpret_cast<CandEntry*>(base + o);
  o += align256(sizeof(CandEntry) * kCapCands);
  S.report = reinterpret_cast<abft_fault*>(base + o);
  o += align256(sizeof(abft_fault) * kCapReport);
  S.part = reinterpret_cast<double*>(base + o);
  S.part_elems = part_elems(P);
  return S;
}

}  // namespace abft

using namespace abft;

extern "C" {

const char* abft_last_error(void) { return g_err; }

int32_t abft_version(void) { return 100; }

int64_t abft_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

size_t abft_workspace_bytes(const abft_desc* desc) {
  Plan P;
  if (make_plan(desc, &P) != ABFT_OK) return 0;
  return P.L.total;
}

abft_status abft_workspace_layout(const abft_desc* desc, abft_ws_layout* out) {
  if (!out) return fail(ABFT_ERR_INVALID, "out is NULL");
  Plan P;
  const abft_status st = make_plan(desc, &P);
  if (st != ABFT_OK) return st;
  *out = P.L;
  return ABFT_OK;
}

abft_status abft_encode(const abft_desc* desc, const void* A, const void* B, const void* a_scale,
                        const void* b_scale, void* ws, void* stream) {
  Plan P;
  abft_status st = make_plan(desc, &P);
  if (st != ABFT_OK) return st;
  if (is_empty(P)) return ABFT_OK;
  if (!ws || (P.d.k > 0 && (!A || !B))) return fail(ABFT_ERR_INVALID, "NULL pointer");
  if (ws_misaligned(ws)) return fail(ABFT_ERR_INVALID, "ws must be 256-byte aligned");
  if (P.d.dtype == ABFT_FP8_E4M3 && P.d.k > 0 && (!a_scale || !b_scale))
    return fail(ABFT_ERR_INVALID, "ABFT_FP8_E4M3 needs a_scale and b_scale");
  cudaError_t e = clear_carry(P, ws, static_cast<cudaStream_t>(stream));
  if (e == cudaSuccess)
    e = P.d.dtype == ABFT_F64
            ? launch_encode_f64(P, static_cast<const double*>(A), static_cast<const double*>(B),
                                ws, static_cast<cudaStream_t>(stream))
            : launch_encode_lp(P, A, B, a_scale, b_scale, ws, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? ABFT_OK : cuda_fail(e, "abft_encode");
}

abft_status abft_encode_chained(const abft_desc* desc, const void* A, const void* B,
                                const abft_desc* left_desc, const void* left_ws,
                                const abft_desc* right_desc, const void* right_ws, void* ws,
                                void* stream) {
  if (!left_desc && !right_desc) return abft_encode(desc, A, B, nullptr, nullptr, ws, stream);
  Plan P, PL, PR;
  abft_status st = make_plan(desc, &P);
  if (st != ABFT_OK) return st;
  const abft_desc& d = P.d;
  const bool split = d.dtype == ABFT_BF16X3 || d.dtype == ABFT_BF16X6;
  if (d.dtype != ABFT_F64 && !split)
    return fail(ABFT_ERR_UNSUPPORTED,
                "chained encode: ABFT_F64, ABFT_BF16X3 and ABFT_BF16X6 products only");
  // the earlier product's C is this product's operand: binary64 C for an
  // ABFT_F64 product, binary32 C (any tensor-core dtype) for a split one
  auto c_matches = [&](int dt) { return split ? dt != ABFT_F64 : dt == ABFT_F64; };
  const char* c_msg = split ? "a split product takes the binary32 C of a tensor-core product"
                            : "an ABFT_F64 product takes the binary64 C of an ABFT_F64 product";
  if (left_desc) {
    if ((st = make_plan(left_desc, &PL)) != ABFT_OK) return st;
    if (!c_matches(PL.d.dtype)) return fail(ABFT_ERR_INVALID, "left chain: %s", c_msg);
    if (PL.d.m != d.m || PL.d.n != d.k || PL.d.vb_rows != d.vb_rows)
      return fail(ABFT_ERR_INVALID,
                  "left chain: the earlier product must be m x k with the same vb_rows");
    if (P.bs > 0 && (PL.d.grid_p != d.grid_p || PL.f < P.f))
      return fail(ABFT_ERR_INVALID,
                  "left chain: the earlier product needs the same grid_p and at least grid_f "
                  "block checksums");
    if (d.k > 0 && !left_ws) return fail(ABFT_ERR_INVALID, "left chain: left_ws is NULL");
  }
  if (right_desc) {
    if ((st = make_plan(right_desc, &PR)) != ABFT_OK) return st;
    if (!c_matches(PR.d.dtype)) return fail(ABFT_ERR_INVALID, "right chain: %s", c_msg);
    if (PR.d.m != d.k || PR.d.n != d.n || PR.d.vb_cols != d.vb_cols)
      return fail(ABFT_ERR_INVALID,
                  "right chain: the earlier product must be k x n with the same vb_cols");
    if (d.k > 0 && !right_ws) return fail(ABFT_ERR_INVALID, "right chain: right_ws is NULL");
  }
  if (is_empty(P)) return ABFT_OK;
  if (!ws || (d.k > 0 && (!A || !B))) return fail(ABFT_ERR_INVALID, "NULL pointer");
  if (ws_misaligned(ws) || (left_desc && ws_misaligned(left_ws)) ||
      (right_desc && ws_misaligned(right_ws)))
    return fail(ABFT_ERR_INVALID, "ws, left_ws and right_ws must be 256-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = clear_carry(P, ws, s);
  if (e == cudaSuccess) {
    const Plan* pl = left_desc ? &PL : nullptr;
    const Plan* pr = right_desc ? &PR : nullptr;
    e = split ? launch_encode_lp_chained(P, A, B, ws, pl, left_ws, pr, right_ws, s)
              : launch_encode_f64_chained(P, static_cast<const double*>(A),
                                          static_cast<const double*>(B), ws, pl, left_ws, pr,
                                          right_ws, s);
  }
  return e == cudaSuccess ? ABFT_OK : cuda_fail(e, "abft_encode_chained");
}

abft_status abft_encode_noalloc(const abft_desc* desc, const void* A, const void* B,
                                const void* a_scale, const void* b_scale, void* ws, void* stream) {
  (void)a_scale;
  (void)b_scale;
  Plan P;
  abft_status st = make_plan(desc, &P);
  if (st != ABFT_OK) return st;
  if (P.d.dtype != ABFT_F64)
    return fail(ABFT_ERR_UNSUPPORTED, "abft_encode_noalloc supports ABFT_F64 only");
  const size_t need = sizeof(double) * part_elems(P);
  if (need > static_encode_part_bytes())
    return fail(ABFT_ERR_INVALID,
                "abft_encode_noalloc: this problem needs %zu bytes of encode scratch, above the "
                "static maximum of %zu bytes; use abft_encode with a full workspace",
                need, static_encode_part_bytes());
  if (is_empty(P)) return ABFT_OK;
  if (!ws || (P.d.k > 0 && (!A || !B))) return fail(ABFT_ERR_INVALID, "NULL pointer");
  if (ws_misaligned(ws)) return fail(ABFT_ERR_INVALID, "ws must be 256-byte aligned");
  cudaError_t e = clear_carry(P, ws, static_cast<cudaStream_t>(stream));
  if (e == cudaSuccess)
    e = launch_encode_f64_noalloc(P, static_cast<const double*>(A), static_cast<const double*>(B),
                                  ws, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? ABFT_OK : cuda_fail(e, "abft_encode_noalloc");
}

static abft_status gemm_common(const abft_desc* desc, const void* A, const void* B, void* C,
                               void* ws, bool checksums, void* stream) {
  Plan P;
  abft_status st = make_plan(desc, &P);
  if (st != ABFT_OK) return st;
  if (is_empty(P)) return ABFT_OK;
  if (!C || ((checksums || P.d.dtype == ABFT_BF16X3 || P.d.dtype == ABFT_BF16X6 ||
               P.d.dtype == ABFT_FP8_E4M3) && !ws) ||
      (P.d.k > 0 && (!A || !B)))
    return fail(ABFT_ERR_INVALID, "NULL pointer");
  if (ws && ws_misaligned(ws)) return fail(ABFT_ERR_INVALID, "ws must be 256-byte aligned");
  cudaError_t e;
  if (P.d.dtype == ABFT_F64) {
    e = launch_gemm_f64(P, static_cast<const double*>(A), static_cast<const double*>(B),
                        static_cast<double*>(C), ws, checksums, static_cast<cudaStream_t>(stream));
  } else {
    if (P.d.dtype == ABFT_BF16 && ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15))
      return fail(ABFT_ERR_INVALID, "bf16 operands must be 16-byte aligned");
    e = launch_gemm_lp(P, A, B, static_cast<float*>(C), ws, checksums,
                       static_cast<cudaStream_t>(stream));
  }
  return e == cudaSuccess ? ABFT_OK : cuda_fail(e, checksums ? "abft_gemm" : "abft_gemm_plain");
}

abft_status abft_gemm(const abft_desc* desc, const void* A, const void* B, const void* a_scale,
                      const void* b_scale, void* C, void* ws, void* stream) {
  (void)a_scale;
  (void)b_scale;
  return gemm_common(desc, A, B, C, ws, true, stream);
}

abft_status abft_gemm_plain(const abft_desc* desc, const void* A, const void* B,
                            const void* a_scale, const void* b_scale, void* C, void* ws,
                            void* stream) {
  (void)a_scale;
  (void)b_scale;
  return gemm_common(desc, A, B, C, ws, false, stream);
}

abft_status abft_set_epilogue_faults(const abft_desc* desc, void* ws, const int64_t* rows,
                                     const int64_t* cols, const int32_t* bits, int32_t count,
                                     void* stream) {
  Plan P;
  abft_status st = make_plan(desc, &P);
  if (st != ABFT_OK) return st;
  if (P.d.dtype == ABFT_F64)
    return fail(ABFT_ERR_UNSUPPORTED, "epilogue fault injection needs a tensor-core dtype");
  if (!ws || count < 0 || count > kMaxInject || (count > 0 && (!rows || !cols || !bits)))
    return fail(ABFT_ERR_INVALID, "bad injection list (at most %d entries)", kMaxInject);
  for (int t = 0; t < count; ++t)
    if (rows[t] < 0 || rows[t] >= P.d.m || cols[t] < 0 || cols[t] >= P.d.n || bits[t] < 0 ||
        bits[t] > 31)
      return fail(ABFT_ERR_INVALID, "injection %d outside C or the fp32 element", t);
  const cudaError_t e =
      launch_set_inject(P, ws, rows, cols, bits, count, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? ABFT_OK : cuda_fail(e, "abft_set_epilogue_faults");
}

abft_status abft_verify_correct(const abft_desc* desc, void* C, void* ws, int32_t reread_C,
                                const int32_t* erased_blocks, int32_t n_erased, abft_fault* report,
                                int32_t max_reports, int32_t* n_reports, void* stream) {
  Plan P;
  abft_status st = make_plan(desc, &P);
  if (st != ABFT_OK) return st;
  if (n_reports) *n_reports = 0;
  if (max_reports < 0 || (max_reports > 0 && !report))
    return fail(ABFT_ERR_INVALID, "report buffer");
  if (n_erased < 0 || n_erased > kMaxErased || (n_erased > 0 && !erased_blocks))
    return fail(ABFT_ERR_INVALID, "n_erased must be in [0, %d]", kMaxErased);
  Erased er{};
  er.n = n_erased;
  for (int t = 0; t < n_erased; ++t) {
    const int bi = erased_blocks[2 * t], bj = erased_blocks[2 * t + 1];
    if (P.bs == 0 || bi < 0 || bj < 0 || bi >= P.d.grid_p || bj >= P.d.grid_q)
      return fail(ABFT_ERR_INVALID, "erased block (%d, %d) outside the erasure grid", bi, bj);
    er.bi[t] = bi;
    er.bj[t] = bj;
  }
  if (is_empty(P)) return ABFT_OK;
  if (!C || !ws) return fail(ABFT_ERR_INVALID, "NULL pointer");
  if (ws_misaligned(ws)) return fail(ABFT_ERR_INVALID, "ws must be 256-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Scratch S = scratch_view(P, ws);
  cudaError_t e = cudaMemsetAsync(S.cnt, 0, sizeof(int32_t) * kNumCleared, s);
  if (e != cudaSuccess) return cuda_fail(e, "abft_verify_correct memset");
  e = launch_verify(P, C, ws, er, reread_C != 0 || !P.fused, s);
  if (e != cudaSuccess) return cuda_fail(e, "abft_verify_correct launch");
  int32_t cnt[kNumCounters];
  e = cudaMemcpyAsync(cnt, S.cnt, sizeof cnt, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "abft_verify_correct");
  // status words of this workspace's last product and last encode
  if (P.d.dtype != ABFT_F64 && cnt[kCntTimeout])
    return fail(ABFT_ERR_TIMEOUT,
                "the tensor-core product on this workspace gave up waiting (bounded wait); C and "
                "its checksums are incomplete and were not corrected");
  if (P.d.dtype == ABFT_FP8_E4M3 && cnt[kCntFp8Inexact])
    return fail(ABFT_ERR_INVALID,
                "an e4m3 value times its block scale is not exact in bf16: the block scales "
                "must be powers of two (and the operands finite)");
  const int total = cnt[kCntReport];
  const int stored = std::min(total, kCapReport);
  std::vector<abft_fault> rep((size_t)stored);
  if (stored > 0) {
    e = cudaMemcpyAsync(rep.data(), S.report, sizeof(abft_fault) * stored, cudaMemcpyDeviceToHost,
                        s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "abft_verify_correct report");
  }
  std::sort(rep.begin(), rep.end(), [](const abft_fault& x, const abft_fault& y) {
    if (x.row != y.row) return x.row < y.row;
    if (x.col != y.col) return x.col < y.col;
    return x.kind < y.kind;
  });
  bool uncorrectable = cnt[kCntOverflow] != 0 || total > kCapReport;
  for (const abft_fault& f : rep) uncorrectable |= f.kind == ABFT_KIND_UNCORRECTABLE;
  const int nout = std::min(stored, max_reports);
  for (int t = 0; t < nout; ++t) report[t] = rep[(size_t)t];
  if (n_reports) *n_reports = total;
  if (cnt[kCntOverflow])
    return fail(ABFT_ERR_UNCORRECTABLE, "too many flagged lines (%d column, %d row)",
                cnt[kCntColFlags], cnt[kCntRowFlags]);
  if (uncorrectable) return fail(ABFT_ERR_UNCORRECTABLE, "flagged lines could not be corrected");
  return ABFT_OK;
}

// Inverse of the t x t matrix M[l][u] = block_coef(l, rows[u], p) (Gauss-Jordan
// with partial pivoting, binary64).  False when it is singular (repeated rows).
static bool invert_block_coefs(const int* rows, int t, int p, double* inv) {
  double a[kMaxBlockChecksums][2 * kMaxBlockChecksums];
  for (int l = 0; l < t; ++l)
    for (int u = 0; u < 2 * t; ++u)
      a[l][u] = u < t ? block_coef(l, rows[u], p) : (u - t == l ? 1.0 : 0.0);
  for (int c = 0; c < t; ++c) {
    int piv = c;
    for (int i = c + 1; i < t; ++i)
      if (fabs(a[i][c]) > fabs(a[piv][c])) piv = i;
    if (!(fabs(a[piv][c]) > 0.0)) return false;
    for (int x = 0; x < 2 * t; ++x) std::swap(a[c][x], a[piv][x]);
    const double d = a[c][c];
    for (int x = 0; x < 2 * t; ++x) a[c][x] /= d;
    for (int i = 0; i < t; ++i)
      if (i != c) {
        const double f = a[i][c];
        for (int x = 0; x < 2 * t; ++x) a[i][x] -= f * a[c][x];
      }
  }
  for (int u = 0; u < t; ++u)
    for (int l = 0; l < t; ++l) inv[u * t + l] = a[u][t + l];
  return true;
}

abft_status abft_recover_blocks(const abft_desc* desc, void* C, void* ws, const int32_t* blocks,
                                int32_t n_blocks, abft_fault* report, void* stream) {
  Plan P;
  abft_status st = make_plan(desc, &P);
  if (st != ABFT_OK) return st;
  if (P.bs == 0) return fail(ABFT_ERR_INVALID, "no erasure grid in the descriptor");
  if (n_blocks < 0 || n_blocks > kMaxErased || (n_blocks > 0 && !blocks))
    return fail(ABFT_ERR_INVALID, "n_blocks must be in [0, %d]", kMaxErased);
  for (int u = 0; u < n_blocks; ++u) {
    const int bi = blocks[2 * u], bj = blocks[2 * u + 1];
    if (bi < 0 || bj < 0 || bi >= P.d.grid_p || bj >= P.d.grid_q)
      return fail(ABFT_ERR_INVALID, "block (%d, %d) outside the erasure grid", bi, bj);
    for (int v = 0; v < u; ++v)
      if (blocks[2 * v] == bi && blocks[2 * v + 1] == bj)
        return fail(ABFT_ERR_INVALID, "block (%d, %d) listed twice", bi, bj);
  }
  // group by block column; more erasures in a column than block checksums
  // cannot be rebuilt
  std::vector<int> cols;
  for (int u = 0; u < n_blocks; ++u)
    if (std::find(cols.begin(), cols.end(), blocks[2 * u + 1]) == cols.end())
      cols.push_back(blocks[2 * u + 1]);
  for (int bj : cols) {
    int t = 0;
    for (int u = 0; u < n_blocks; ++u) t += blocks[2 * u + 1] == bj;
    if (t > P.f)
      return fail(ABFT_ERR_UNCORRECTABLE,
                  "%d erased blocks in block column %d, more than the %d block checksums", t, bj,
                  P.f);
  }
  if (n_blocks == 0) return ABFT_OK;
  if (!C || !ws) return fail(ABFT_ERR_INVALID, "NULL pointer");
  if (ws_misaligned(ws)) return fail(ABFT_ERR_INVALID, "ws must be 256-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Scratch S = scratch_view(P, ws);
  cudaError_t e = cudaMemsetAsync(S.cnt + kCntRecoverFlagged, 0, sizeof(int32_t), s);
  for (int bj : cols) {
    if (e != cudaSuccess) break;
    int rows[kMaxBlockChecksums], t = 0;
    for (int u = 0; u < n_blocks; ++u)
      if (blocks[2 * u + 1] == bj) rows[t++] = blocks[2 * u];
    double minv[kMaxBlockChecksums * kMaxBlockChecksums];
    if (!invert_block_coefs(rows, t, P.d.grid_p, minv))
      return fail(ABFT_ERR_INVALID, "singular block-checksum system in block column %d", bj);
    e = launch_recover(P, C, ws, bj, rows, t, minv, s);
  }
  int32_t cnt[kNumCounters] = {};
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(cnt, S.cnt, sizeof cnt, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "abft_recover_blocks");
  if (P.d.dtype != ABFT_F64 && cnt[kCntTimeout])
    return fail(ABFT_ERR_TIMEOUT,
                "the tensor-core product on this workspace gave up waiting (bounded wait); its "
                "block checksums are incomplete and nothing was rebuilt");
  const int32_t nfl = cnt[kCntRecoverFlagged];
  if (report)
    for (int u = 0; u < n_blocks; ++u) {
      abft_fault f{};
      f.row = (int32_t)(blocks[2 * u] * P.bs);
      f.col = (int32_t)(blocks[2 * u + 1] * P.bc);
      f.kind = ABFT_KIND_BLOCK_RECOVERED;
      f.side = 2;
      f.r_e = (double)nfl;
      report[u] = f;
    }
  if (nfl) return fail(ABFT_ERR_UNCORRECTABLE, "rebuilt blocks fail %d column checks", nfl);
  return ABFT_OK;
}

abft_status abft_recover_block(const abft_desc* desc, void* C, void* ws, int32_t bi, int32_t bj,
                               abft_fault* report_entry, void* stream) {
  const int32_t blk[2] = {bi, bj};
  return abft_recover_blocks(desc, C, ws, blk, 1, report_entry, stream);
}

abft_status abft_block_partial(const abft_desc* desc, const void* C, const void* ws,
                               int32_t bi_skip, int32_t bj, int32_t with_checksum, double* out,
                               void* stream) {
  Plan P;
  abft_status st = make_plan(desc, &P);
  if (st != ABFT_OK) return st;
  if (P.bs == 0) return fail(ABFT_ERR_INVALID, "no erasure grid in the descriptor");
  if (bj < 0 || bj >= P.d.grid_q || bi_skip < -1 || bi_skip >= P.d.grid_p)
    return fail(ABFT_ERR_INVALID, "block column %d / skipped block row %d outside the grid", bj,
                bi_skip);
  if (!C || !out || (with_checksum && !ws)) return fail(ABFT_ERR_INVALID, "NULL pointer");
  if (ws && ws_misaligned(ws)) return fail(ABFT_ERR_INVALID, "ws must be 256-byte aligned");
  const cudaError_t e = launch_block_partial(P, C, ws, bi_skip, bj, with_checksum != 0, out,
                                             static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? ABFT_OK : cuda_fail(e, "abft_block_partial");
}

abft_status abft_block_restore(const abft_desc* desc, void* C, void* ws, int32_t bi, int32_t bj,
                               const double* sum, abft_fault* report_entry, void* stream) {
  Plan P;
  abft_status st = make_plan(desc, &P);
  if (st != ABFT_OK) return st;
  if (P.bs == 0) return fail(ABFT_ERR_INVALID, "no erasure grid in the descriptor");
  if (bi < 0 || bj < 0 || bi >= P.d.grid_p || bj >= P.d.grid_q)
    return fail(ABFT_ERR_INVALID, "block (%d, %d) outside the erasure grid", bi, bj);
  if (!C || !ws || !sum) return fail(ABFT_ERR_INVALID, "NULL pointer");
  if (ws_misaligned(ws)) return fail(ABFT_ERR_INVALID, "ws must be 256-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Scratch S = scratch_view(P, ws);
  cudaError_t e = cudaMemsetAsync(S.cnt + kCntRecoverFlagged, 0, sizeof(int32_t), s);
  if (e == cudaSuccess) e = launch_block_restore(P, C, ws, bi, bj, sum, s);
  int32_t cnt[kNumCounters] = {};
  if (e == cudaSuccess) e = cudaMemcpyAsync(cnt, S.cnt, sizeof cnt, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "abft_block_restore");
  if (P.d.dtype != ABFT_F64 && cnt[kCntTimeout])
    return fail(ABFT_ERR_TIMEOUT,
                "the tensor-core product on this workspace gave up waiting (bounded wait); "
                "nothing was written");
  const int32_t nfl = cnt[kCntRecoverFlagged];
  if (report_entry) {
    abft_fault f{};
    f.row = (int32_t)(bi * P.bs);
    f.col = (int32_t)(bj * P.bc);
    f.kind = ABFT_KIND_BLOCK_RECOVERED;
    f.side = 2;
    f.r_e = (double)nfl;
    *report_entry = f;
  }
  if (nfl) return fail(ABFT_ERR_UNCORRECTABLE, "rebuilt block fails %d column checks", nfl);
  return ABFT_OK;
}

abft_status abft_inject_bitflips(const abft_desc* desc, void* C, const int64_t* rows,
                                 const int64_t* cols, const int32_t* bits, int32_t count,
                                 void* stream) {
  Plan P;
  abft_status st = make_plan(desc, &P);
  if (st != ABFT_OK) return st;
  if (count < 0 || (count > 0 && (!rows || !cols || !bits || !C)))
    return fail(ABFT_ERR_INVALID, "bad flip list");
  const int width = P.d.dtype == ABFT_F64 ? 64 : 32;
  for (int t = 0; t < count; ++t)
    if (rows[t] < 0 || rows[t] >= P.d.m || cols[t] < 0 || cols[t] >= P.d.n || bits[t] < 0 ||
        bits[t] >= width)
      return fail(ABFT_ERR_INVALID, "flip %d outside C or the element width", t);
  if (count == 0) return ABFT_OK;
  const cudaError_t e = launch_inject(P, C, rows, cols, bits, count, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? ABFT_OK : cuda_fail(e, "abft_inject_bitflips");
}

abft_status abft_erase_block(const abft_desc* desc, void* C, int32_t bi, int32_t bj, void* stream) {
  Plan P;
  abft_status st = make_plan(desc, &P);
  if (st != ABFT_OK) return st;
  if (P.bs == 0) return fail(ABFT_ERR_INVALID, "no erasure grid in the descriptor");
  if (bi < 0 || bj < 0 || bi >= P.d.grid_p || bj >= P.d.grid_q || !C)
    return fail(ABFT_ERR_INVALID, "block (%d, %d) outside the erasure grid", bi, bj);
  const cudaError_t e = launch_erase(P, C, bi, bj, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? ABFT_OK : cuda_fail(e, "abft_erase_block");
}

}  // extern "C"
