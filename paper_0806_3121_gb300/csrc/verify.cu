// Detect / locate / correct and erasure recovery (sections 1, 2.1 and 2.2 of
// the paper: the consistency of (AB)_F detects, localizes and corrects
// errors; a lost part is the checksum minus the surviving parts).
//
// Pipeline of one verify call, all on the device:
//   k_col_check   one thread per column line (verify block I, column j):
//                 binary64 sums e^T C_I[:,j], w^T C_I[:,j], non-finite count,
//                 residuals against E, threshold test, append if flagged.
//   k_row_check   one warp per row line (row i, verify block J), against F.
//   k_locate_correct  one CTA: candidates from the flagged lines (single
//                 non-finite element, or the weighted/unweighted residual
//                 ratio), bitonic sort + merge, choice of a correcting line,
//                 recomputation in binary64, re-check of the touched lines,
//                 report entries.
// Recovery: k_recover rebuilds an erased block from S = sum_I C_I, then
// k_col_check (count mode) re-checks the rebuilt block.
#include <math.h>

#include "internal.cuh"

namespace abft {
namespace {

constexpr int kThreads = 256;
constexpr int kLocThreads = 512;

struct CheckArgs {
  const void* C;
  int64_t ldc, m, n;
  const double* E;  // R x n, row 2I = e-checksum, 2I+1 = w-checksum, then S
  const double* F;  // m x Cc
  const double* nArow;
  const double* nAblk;
  const double* nBcol;
  const double* nBblk;
  const double* carA;  // carried-checksum deviation bounds (zero unless chained)
  const double* carB;
  int vb_r, vb_c, er, ec;
  int64_t nvr, nvc, Cc, bs, bc;
  double s, f1c, f2c, f1r, f2r;
  Erased erased;
  FlagEntry* colf;
  FlagEntry* rowf;
  int32_t* cnt;
  abft_fault* report;
  CandEntry* cand;
  // status word of the workspace's last tensor-core product (nullptr for
  // binary64): when that product timed out, C is incomplete and nothing is
  // located or corrected
  const int32_t* timeout;
};

template <typename TC>
__device__ __forceinline__ double ld(const void* C, int64_t idx) {
  return (double)static_cast<const TC*>(C)[idx];
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ int warp_isum(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ long long warp_min(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w < v ? w : v;
  }
  return v;
}

__device__ __forceinline__ bool touches_erased(const Erased& e, int64_t bs, int64_t bc, int64_t i0,
                                               int64_t i1, int64_t j0, int64_t j1) {
  for (int t = 0; t < e.n; ++t) {
    const int64_t r0 = (int64_t)e.bi[t] * bs, c0 = (int64_t)e.bj[t] * bc;
    if (i0 < r0 + bs && r0 < i1 && j0 < c0 + bc && c0 < j1) return true;
  }
  return false;
}

// Flag rule: not (|r_e| <= tau_e and |r_w| <= tau_w); NaN residuals fail it.
__device__ __forceinline__ bool is_flagged(double re, double rw, double te, double tw) {
  return !(fabs(re) <= te && fabs(rw) <= tw);
}

__device__ __forceinline__ void col_taus(const CheckArgs& a, int64_t I, int64_t j, double& te,
                                         double& tw) {
  const double nb = a.nBcol[j];
  te = a.s * nb * (a.f1c * a.nAblk[4 * I + 0] + a.f2c * a.nAblk[4 * I + 2] + a.carA[2 * I]);
  tw = a.s * nb * (a.f1c * a.nAblk[4 * I + 1] + a.f2c * a.nAblk[4 * I + 3] + a.carA[2 * I + 1]);
}
__device__ __forceinline__ void row_taus(const CheckArgs& a, int64_t i, int64_t J, double& te,
                                         double& tw) {
  const double na = a.nArow[i];
  te = a.s * na * (a.f1r * a.nBblk[4 * J + 0] + a.f2r * a.nBblk[4 * J + 2] + a.carB[2 * J]);
  tw = a.s * na * (a.f1r * a.nBblk[4 * J + 1] + a.f2r * a.nBblk[4 * J + 3] + a.carB[2 * J + 1]);
}

// Observed block sums run in the element type of C: binary64 for a binary64
// C, binary32 for a binary32 C (whose rounding the thresholds carry as u_sum).
template <typename TC>
__device__ __forceinline__ TC fma_t(TC a, TC b, TC c);
template <>
__device__ __forceinline__ double fma_t<double>(double a, double b, double c) { return fma(a, b, c); }
template <>
__device__ __forceinline__ float fma_t<float>(float a, float b, float c) { return fmaf(a, b, c); }

template <typename TC>
__device__ __forceinline__ TC warp_sum_t(TC v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Residuals of column line (I, j).  Returns the non-finite count.
template <typename TC>
__device__ int col_line(const CheckArgs& a, int64_t I, int64_t j, double& re, double& rw,
                        double& te, double& tw) {
  const int64_t i0 = I * a.vb_r, i1 = min(i0 + (int64_t)a.vb_r, a.m);
  const TC sc = (TC)scalbn(1.0, -a.er);
  const TC* C = static_cast<const TC*>(a.C);
  TC se = 0, sw = 0;
  int nf = 0;
  const TC* p = C + i0 * a.ldc + j;
  const int len = (int)(i1 - i0);
#pragma unroll 4
  for (int t = 0; t < len; ++t) {
    const TC x = p[(int64_t)t * a.ldc];
    se += x;
    sw = fma_t<TC>((TC)(t + 1) * sc, x, sw);
    nf += isfinite(x) ? 0 : 1;
  }
  re = (double)se - a.E[(2 * I) * a.n + j];
  rw = (double)sw - a.E[(2 * I + 1) * a.n + j];
  col_taus(a, I, j, te, tw);
  return nf;
}

// The same computed by one warp (lanes split the rows; sums in the element
// type, then added across the lanes); residuals and thresholds valid in every
// lane.
template <typename TC>
__device__ int col_line_warp(const CheckArgs& a, int64_t I, int64_t j, double& re, double& rw,
                             double& te, double& tw) {
  const int lane = threadIdx.x & 31;
  const int64_t i0 = I * a.vb_r, i1 = min(i0 + (int64_t)a.vb_r, a.m);
  const TC sc = (TC)scalbn(1.0, -a.er);
  const TC* C = static_cast<const TC*>(a.C);
  TC se = 0, sw = 0;
  int nf = 0;
  const int len = (int)(i1 - i0);
  for (int t = lane; t < len; t += 32) {
    const TC x = C[(i0 + t) * a.ldc + j];
    se += x;
    sw = fma_t<TC>((TC)(t + 1) * sc, x, sw);
    nf += isfinite(x) ? 0 : 1;
  }
  se = warp_sum_t<TC>(se);
  sw = warp_sum_t<TC>(sw);
  nf = warp_isum(nf);
  re = (double)se - a.E[(2 * I) * a.n + j];
  rw = (double)sw - a.E[(2 * I + 1) * a.n + j];
  col_taus(a, I, j, te, tw);
  return nf;
}

// Residuals of row line (i, J) computed by one warp; the sums and the
// non-finite count are valid in every lane, the residuals and thresholds in
// lane 0 only (binary64 work done once per line).
template <typename TC>
__device__ int row_line_warp(const CheckArgs& a, int64_t i, int64_t J, double& re, double& rw,
                             double& te, double& tw) {
  const int lane = threadIdx.x & 31;
  const int64_t j0 = J * a.vb_c, j1 = min(j0 + (int64_t)a.vb_c, a.n);
  const TC sc = (TC)scalbn(1.0, -a.ec);
  const TC* C = static_cast<const TC*>(a.C);
  TC se = 0, sw = 0;
  int nf = 0;
  const TC* p = C + i * a.ldc + j0;
  const int len = (int)(j1 - j0);
  for (int t = lane; t < len; t += 32) {
    const TC x = p[t];
    se += x;
    sw = fma_t<TC>((TC)(t + 1) * sc, x, sw);
    nf += isfinite(x) ? 0 : 1;
  }
  se = warp_sum_t<TC>(se);
  sw = warp_sum_t<TC>(sw);
  nf = warp_isum(nf);
  re = rw = te = tw = 0.0;
  if (lane == 0) {
    re = (double)se - a.F[i * a.Cc + 2 * J];
    rw = (double)sw - a.F[i * a.Cc + 2 * J + 1];
    row_taus(a, i, J, te, tw);
  }
  return nf;
}

// Column lines [I_begin, I_end) x [j_begin, j_end).  mode 0: append flagged
// lines to colf (skipping erased blocks); mode 1: only count them in
// cnt[kCntRecoverFlagged].  Grid (ceil((j_end-j_begin)/256), <= 65535).
template <typename TC>
__global__ void __launch_bounds__(kThreads) k_col_check(const CheckArgs a, int64_t j_begin,
                                                        int64_t j_end, int64_t I_begin,
                                                        int64_t I_end, int mode) {
  const int64_t j = j_begin + (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (j >= j_end) return;
  for (int64_t I = I_begin + blockIdx.y; I < I_end; I += gridDim.y) {
    const int64_t i0 = I * a.vb_r, i1 = min(i0 + (int64_t)a.vb_r, a.m);
    if (mode == 0 && touches_erased(a.erased, a.bs, a.bc, i0, i1, j, j + 1)) continue;
    double re, rw, te, tw;
    const int nf = col_line<TC>(a, I, j, re, rw, te, tw);
    if (nf == 0 && !is_flagged(re, rw, te, tw)) continue;
    if (mode == 1) {
      atomicAdd(&a.cnt[kCntRecoverFlagged], 1);
      continue;
    }
    const int slot = atomicAdd(&a.cnt[kCntColFlags], 1);
    if (slot < kCapFlags) a.colf[slot] = FlagEntry{(int32_t)I, (int32_t)j, nf, 0, re, rw};
  }
}

template <typename TC>
__global__ void __launch_bounds__(kThreads) k_row_check(const CheckArgs a) {
  const int64_t gw = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
  if (gw >= a.m * a.nvc) return;
  const int64_t i = gw / a.nvc, J = gw % a.nvc;
  const int64_t j0 = J * a.vb_c, j1 = min(j0 + (int64_t)a.vb_c, a.n);
  if (touches_erased(a.erased, a.bs, a.bc, i, i + 1, j0, j1)) return;
  double re, rw, te, tw;
  const int nf = row_line_warp<TC>(a, i, J, re, rw, te, tw);
  if ((threadIdx.x & 31) != 0) return;
  if (nf == 0 && !is_flagged(re, rw, te, tw)) return;
  const int slot = atomicAdd(&a.cnt[kCntRowFlags], 1);
  if (slot < kCapFlags) a.rowf[slot] = FlagEntry{(int32_t)i, (int32_t)J, nf, 0, re, rw};
}

// Screen of the fused checks: a line whose binary32 evaluation passes with a
// margin is one the binary64 rule passes, so only the others are evaluated in
// binary64 (GB300's FP64 pipe is narrow: the binary64 sums of every line took
// most of the verify).  With s the binary32 sum of the observed partials (nt of
// them, absolute sum b), e the expected checksum rounded to binary32 and r the
// binary32 residual s - e: the binary64 residual is at most
// |r| + (nt + 2) u32 (b + |e| + |r|) in magnitude (u32 = 2^-24; the partials'
// sum, e's rounding and the subtraction), and the binary32 threshold t is
// within a few u32 of the binary64 one, so |r| + (nt + 2) u32 (b + |e| + |r|)
// <= 0.99 t implies the binary64 test passes.  Non-finite or overflowing
// values never pass the screen.
__device__ __forceinline__ bool fused_screen(float sum, float e, float b, float t, float slack) {
  const float r = sum - e;
  const float lhs = fabsf(r) + slack * (b + fabsf(e) + fabsf(r));
  return lhs < 3.0e38f && t < 3.0e38f && lhs <= 0.99f * t;  // false for NaN
}
constexpr float kU32 = 5.9604645e-8f;  // 2^-24

// Column lines from the observed partial sums the product's epilogue wrote
// (one per 32 rows): obs[(block*2 + 0|1)*n + j].  Verify blocks span whole
// 32-row blocks.  A non-finite observed sum marks the line non-finite (the
// locate step then scans C for it).  The lines that pass the binary32 screen
// are done; the others are decided by the binary64 rule.
__global__ void __launch_bounds__(kThreads) k_col_fused(const CheckArgs a, const float* obs,
                                                        int64_t ntr) {
  __shared__ float tI[2];  // the verify block's threshold factors (binary32)
  const int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const bool jv = j < a.n;
  const int64_t tpb = a.vb_r / 32;  // 32-row blocks per verify block
  const float nbj = jv ? (float)a.nBcol[j] : 0.f;
  const float slack = (float)(tpb + 2) * kU32;
  for (int64_t I = blockIdx.y; I < a.nvr; I += gridDim.y) {
    __syncthreads();  // every thread has read the previous tI
    if (threadIdx.x == 0) {
      tI[0] = (float)(a.s * (a.f1c * a.nAblk[4 * I + 0] + a.f2c * a.nAblk[4 * I + 2] + a.carA[2 * I]));
      tI[1] = (float)(a.s * (a.f1c * a.nAblk[4 * I + 1] + a.f2c * a.nAblk[4 * I + 3] +
                             a.carA[2 * I + 1]));
    }
    __syncthreads();
    if (!jv) continue;
    const int64_t i0 = I * a.vb_r, i1 = min(i0 + (int64_t)a.vb_r, a.m);
    if (touches_erased(a.erased, a.bs, a.bc, i0, i1, j, j + 1)) continue;
    const int64_t tr0 = I * tpb, tr1 = min((I + 1) * tpb, ntr);
    float s0 = 0.f, s1 = 0.f, b0 = 0.f, b1 = 0.f;
    for (int64_t tr = tr0; tr < tr1; ++tr) {
      const float x0 = obs[(tr * 2 + 0) * a.n + j], x1 = obs[(tr * 2 + 1) * a.n + j];
      s0 += x0;
      s1 += x1;
      b0 += fabsf(x0);
      b1 += fabsf(x1);
    }
    const double E0 = a.E[(2 * I) * a.n + j], E1 = a.E[(2 * I + 1) * a.n + j];
    if (fused_screen(s0, (float)E0, b0, nbj * tI[0], slack) &&
        fused_screen(s1, (float)E1, b1, nbj * tI[1], slack))
      continue;
    double se = 0.0, sw = 0.0;
    for (int64_t tr = tr0; tr < tr1; ++tr) {
      se += (double)obs[(tr * 2 + 0) * a.n + j];
      sw += (double)obs[(tr * 2 + 1) * a.n + j];
    }
    const int nf = (isfinite(se) && isfinite(sw)) ? 0 : 1;
    const double re = se - E0, rw = sw - E1;
    double te, tw;
    col_taus(a, I, j, te, tw);
    if (nf == 0 && !is_flagged(re, rw, te, tw)) continue;
    const int slot = atomicAdd(&a.cnt[kCntColFlags], 1);
    if (slot < kCapFlags) a.colf[slot] = FlagEntry{(int32_t)I, (int32_t)j, nf, 0, re, rw};
  }
}

// Row lines from the per-row partial sums over column groups of g columns:
// obs[(i*ngrp + group)*2 + 0|1].  One thread per (row, verify block); the
// verify blocks' threshold factors in binary32 in shared memory (up to
// kRowTauSmem blocks; more: computed per line), then the same screen.
constexpr int kRowTauSmem = 2048;
__global__ void __launch_bounds__(kThreads) k_row_fused(const CheckArgs a, const float* obs,
                                                        int64_t g, int64_t ngrp) {
  __shared__ float tJ[2 * kRowTauSmem];
  const bool smem_tau = a.nvc <= kRowTauSmem;
  if (smem_tau) {
    for (int64_t J = threadIdx.x; J < a.nvc; J += kThreads) {
      tJ[2 * J] = (float)(a.s * (a.f1r * a.nBblk[4 * J + 0] + a.f2r * a.nBblk[4 * J + 2] +
                                 a.carB[2 * J]));
      tJ[2 * J + 1] = (float)(a.s * (a.f1r * a.nBblk[4 * J + 1] + a.f2r * a.nBblk[4 * J + 3] +
                                     a.carB[2 * J + 1]));
    }
    __syncthreads();
  }
  const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (t >= a.m * a.nvc) return;
  const int64_t i = t / a.nvc, J = t % a.nvc;
  const int64_t j0 = J * a.vb_c, j1 = min(j0 + (int64_t)a.vb_c, a.n);
  if (touches_erased(a.erased, a.bs, a.bc, i, i + 1, j0, j1)) return;
  const int64_t g0 = j0 / g, g1 = min(cdiv(j1, g), ngrp);
  const double F0 = a.F[i * a.Cc + 2 * J], F1 = a.F[i * a.Cc + 2 * J + 1];
  if (smem_tau) {
    float s0 = 0.f, s1 = 0.f, b0 = 0.f, b1 = 0.f;
    for (int64_t gr = g0; gr < g1; ++gr) {
      const float x0 = obs[(i * ngrp + gr) * 2 + 0], x1 = obs[(i * ngrp + gr) * 2 + 1];
      s0 += x0;
      s1 += x1;
      b0 += fabsf(x0);
      b1 += fabsf(x1);
    }
    const float na = (float)a.nArow[i], slack = (float)(g1 - g0 + 2) * kU32;
    if (fused_screen(s0, (float)F0, b0, na * tJ[2 * J], slack) &&
        fused_screen(s1, (float)F1, b1, na * tJ[2 * J + 1], slack))
      return;
  }
  double se = 0.0, sw = 0.0;
  for (int64_t gr = g0; gr < g1; ++gr) {
    se += (double)obs[(i * ngrp + gr) * 2 + 0];
    sw += (double)obs[(i * ngrp + gr) * 2 + 1];
  }
  const int nf = (isfinite(se) && isfinite(sw)) ? 0 : 1;
  const double re = se - F0, rw = sw - F1;
  double te, tw;
  row_taus(a, i, J, te, tw);
  if (nf == 0 && !is_flagged(re, rw, te, tw)) return;
  const int slot = atomicAdd(&a.cnt[kCntRowFlags], 1);
  if (slot < kCapFlags) a.rowf[slot] = FlagEntry{(int32_t)i, (int32_t)J, nf, 0, re, rw};
}

// Position (0-based) of a single error inside a line of len elements from
// rho = 2^e r_w / r_e, accepted within 0.25 of an integer in [1, len].
__device__ __forceinline__ int64_t ratio_position(double re, double rw, int e, int64_t len) {
  if (!(re != 0.0) || !isfinite(re) || !isfinite(rw)) return -1;
  const double rho = scalbn(rw / re, e);
  if (!isfinite(rho)) return -1;
  const double r = rint(rho);
  if (!(fabs(rho - r) <= 0.25) || r < 1.0 || r > (double)len) return -1;
  return (int64_t)r - 1;
}

// Access to the problem (or problems) a locate pass works on: geometry,
// elements of C, expected checksums, re-checks of lines and the sort keys of
// candidate elements (problem, row, column, side).
struct Geo {
  int64_t m, n, vb_r, vb_c;
  int er, ec;
};

template <typename TC>
struct SinglePol {
  CheckArgs a;
  __device__ __forceinline__ Geo geo(int) const {
    return Geo{a.m, a.n, a.vb_r, a.vb_c, a.er, a.ec};
  }
  __device__ __forceinline__ double ldc(int, int64_t i, int64_t j) const {
    return ld<TC>(a.C, i * a.ldc + j);
  }
  // Stores v rounded to C's type; returns the old value minus the new one.
  __device__ __forceinline__ double stc(int, int64_t i, int64_t j, double v) const {
    TC* Cp = static_cast<TC*>(const_cast<void*>(a.C));
    const TC old = Cp[i * a.ldc + j], nv = (TC)v;
    Cp[i * a.ldc + j] = nv;
    return (double)old - (double)nv;
  }
  __device__ __forceinline__ double expect_col(int, int64_t I, int64_t j) const {
    return a.E[(2 * I) * a.n + j];
  }
  __device__ __forceinline__ double tau_col(int, int64_t I, int64_t j) const {
    double te, tw;
    col_taus(a, I, j, te, tw);
    return te;
  }
  __device__ __forceinline__ double tau_row(int, int64_t i, int64_t J) const {
    double te, tw;
    row_taus(a, i, J, te, tw);
    return te;
  }
  __device__ __forceinline__ double expect_row(int, int64_t i, int64_t J) const {
    return a.F[i * a.Cc + 2 * J];
  }
  // Warp-wide; the result is valid in every lane.
  __device__ __forceinline__ bool recheck_col(int, int64_t I, int64_t j, double& re,
                                              double& rw) const {
    double te, tw;
    col_line_warp<TC>(a, I, j, re, rw, te, tw);
    return is_flagged(re, rw, te, tw);
  }
  // Warp-wide; the result is valid in lane 0.
  __device__ __forceinline__ bool recheck_row(int, int64_t i, int64_t J, double& re,
                                              double& rw) const {
    double te, tw;
    row_line_warp<TC>(a, i, J, re, rw, te, tw);
    return (threadIdx.x & 31) == 0 && is_flagged(re, rw, te, tw);
  }
  __device__ __forceinline__ uint64_t key(int, int64_t r, int64_t c, int side) const {
    return ((uint64_t)r << 32) | ((uint64_t)c << 1) | (uint64_t)side;
  }
  __device__ __forceinline__ int kp(uint64_t) const { return 0; }
  __device__ __forceinline__ int32_t kr(uint64_t k) const { return (int32_t)(k >> 32); }
  __device__ __forceinline__ int32_t kc(uint64_t k) const {
    return (int32_t)((k >> 1) & 0x7fffffffu);
  }
};

__device__ __forceinline__ void push_report(abft_fault* report, int32_t* cnt, int prob,
                                            int32_t row, int32_t col, int kind, int side,
                                            double delta, double re, double rw) {
  const int slot = atomicAdd(&cnt[kCntReport], 1);
  if (slot < kCapReport) {
    abft_fault f{row, col, kind, side, delta, re, rw};
    f.problem = prob;
    report[slot] = f;
  }
}

// Locate and correct, one CTA: candidates from the flagged lines, bitonic
// sort, merge of duplicates, choice of a correcting line, recomputation in
// binary64, re-check of the touched lines.
template <class Pol>
__device__ __forceinline__ void locate_body(const Pol& A, int32_t* cnt, const FlagEntry* colf,
                                            const FlagEntry* rowf, CandEntry* cand,
                                            abft_fault* report) {
  __shared__ uint64_t keys[kCapCands];
  __shared__ int32_t sidx[kCapCands];
  __shared__ int32_t how[kCapCands];   // -2 duplicate, -1 uncorrectable, 0 column, 1 row
  __shared__ int32_t mkind[kCapCands];
  __shared__ int s_nc;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = kLocThreads / 32;
  if (tid == 0) s_nc = 0;
  __syncthreads();
  const int ncf = cnt[kCntColFlags], nrf = cnt[kCntRowFlags];
  const int ncl = min(ncf, kCapFlags), nrl = min(nrf, kCapFlags);
  if (tid == 0 && (ncf > kCapFlags || nrf > kCapFlags)) cnt[kCntOverflow] = 1;

  // 1. candidates
  for (int L = warp; L < ncl + nrl; L += nwarps) {
    const bool colside = L < ncl;
    const FlagEntry f = colside ? colf[L] : rowf[L - ncl];
    const int p = f.pad;
    const Geo G = A.geo(p);
    int64_t row = -1, col = -1;
    int kind = 0;
    if (colside) {
      const int64_t I = f.a, j = f.b, i0 = I * G.vb_r, i1 = min(i0 + G.vb_r, G.m);
      if (f.nonfin > 0) {
        int c = 0;
        long long pos = LLONG_MAX;
        for (int64_t i = i0 + lane; i < i1; i += 32)
          if (!isfinite(A.ldc(p, i, j))) { ++c; pos = min(pos, (long long)i); }
        c = warp_isum(c);
        pos = warp_min(pos);
        if (c == 1) { row = pos; col = j; kind = ABFT_KIND_NONFINITE_CORRECTED; }
      } else {
        const int64_t t = ratio_position(f.re, f.rw, G.er, i1 - i0);
        if (t >= 0) { row = i0 + t; col = j; kind = ABFT_KIND_CORRECTED; }
      }
    } else {
      const int64_t i = f.a, J = f.b, j0 = J * G.vb_c, j1 = min(j0 + G.vb_c, G.n);
      if (f.nonfin > 0) {
        int c = 0;
        long long pos = LLONG_MAX;
        for (int64_t j = j0 + lane; j < j1; j += 32)
          if (!isfinite(A.ldc(p, i, j))) { ++c; pos = min(pos, (long long)j); }
        c = warp_isum(c);
        pos = warp_min(pos);
        if (c == 1) { row = i; col = pos; kind = ABFT_KIND_NONFINITE_CORRECTED; }
      } else {
        const int64_t t = ratio_position(f.re, f.rw, G.ec, j1 - j0);
        if (t >= 0) { row = i; col = j0 + t; kind = ABFT_KIND_CORRECTED; }
      }
    }
    if (lane == 0 && kind != 0) {
      const int slot = atomicAdd(&s_nc, 1);
      if (slot < kCapCands) {
        CandEntry ce{(int32_t)row, (int32_t)col, kind, colside ? 0 : 1, f.re, f.rw};
        ce.prob = p;
        cand[slot] = ce;
        keys[slot] = A.key(p, row, col, colside ? 0 : 1);
        sidx[slot] = slot;
      }
    }
  }
  __syncthreads();
  const int nc = min(s_nc, kCapCands);
  if (tid == 0 && s_nc > kCapCands) cnt[kCntOverflow] = 1;
  if (tid == 0) cnt[kCntCands] = s_nc;

  // 2. bitonic sort of (key, index), padded to a power of two
  int P2 = 1;
  while (P2 < nc) P2 <<= 1;
  for (int t = nc + tid; t < P2; t += kLocThreads) { keys[t] = ~0ull; sidx[t] = -1; }
  __syncthreads();
  for (int k2 = 2; k2 <= P2; k2 <<= 1) {
    for (int jj = k2 >> 1; jj > 0; jj >>= 1) {
      for (int t = tid; t < P2; t += kLocThreads) {
        const int o = t ^ jj;
        if (o > t) {
          const bool up = (t & k2) == 0;
          if ((keys[t] > keys[o]) == up) {
            const uint64_t kt = keys[t]; keys[t] = keys[o]; keys[o] = kt;
            const int32_t it = sidx[t]; sidx[t] = sidx[o]; sidx[o] = it;
          }
        }
      }
      __syncthreads();
    }
  }

  // 3. merge duplicates (one element can be proposed by its column line and
  //    by its row line; the column entry sorts first and is kept)
  for (int t = tid; t < nc; t += kLocThreads) {
    const bool dup = t > 0 && (keys[t] >> 1) == (keys[t - 1] >> 1);
    how[t] = dup ? -2 : 0;
    int kd = cand[sidx[t]].kind;
    if (!dup && t + 1 < nc && (keys[t + 1] >> 1) == (keys[t] >> 1) &&
        cand[sidx[t + 1]].kind == ABFT_KIND_NONFINITE_CORRECTED)
      kd = ABFT_KIND_NONFINITE_CORRECTED;
    mkind[t] = kd;
  }
  __syncthreads();

  // 4. choose the correcting line: one in which the candidate is alone
  for (int t = tid; t < nc; t += kLocThreads) {
    if (how[t] == -2) continue;
    const int p = A.kp(keys[t]);
    const Geo G = A.geo(p);
    const int32_t r = A.kr(keys[t]), c = A.kc(keys[t]);
    const int64_t I = r / G.vb_r, J = c / G.vb_c;
    int ncol = 0, nrow = 0;
    for (int u = 0; u < nc; ++u) {
      if ((keys[u] >> 1) == ((u > 0) ? (keys[u - 1] >> 1) : ~0ull)) continue;  // duplicate
      if (A.kp(keys[u]) != p) continue;
      const int32_t r2 = A.kr(keys[u]), c2 = A.kc(keys[u]);
      if (c2 == c && r2 / G.vb_r == I) ++ncol;
      if (r2 == r && c2 / G.vb_c == J) ++nrow;
    }
    how[t] = ncol == 1 ? 0 : (nrow == 1 ? 1 : -1);
    // alone in both lines: recompute from the line whose unweighted threshold
    // (the scale of its rounding errors) is smaller; ties take the column
    if (ncol == 1 && nrow == 1 && A.tau_row(p, r, J) < A.tau_col(p, I, c)) how[t] = 1;
  }
  __syncthreads();

  // 5. flagged lines holding no candidate are uncorrectable
  for (int L = tid; L < ncl + nrl; L += kLocThreads) {
    const bool colside = L < ncl;
    const FlagEntry f = colside ? colf[L] : rowf[L - ncl];
    const int p = f.pad;
    const Geo G = A.geo(p);
    bool has = false;
    for (int u = 0; u < nc && !has; ++u) {
      if (how[u] == -2 || A.kp(keys[u]) != p) continue;
      const int32_t r2 = A.kr(keys[u]), c2 = A.kc(keys[u]);
      has = colside ? (c2 == f.b && r2 / G.vb_r == f.a) : (r2 == f.a && c2 / G.vb_c == f.b);
    }
    if (!has) {
      if (colside) push_report(report, cnt, p, -1, f.b, ABFT_KIND_UNCORRECTABLE, 0, 0.0, f.re, f.rw);
      else push_report(report, cnt, p, f.a, -1, ABFT_KIND_UNCORRECTABLE, 1, 0.0, f.re, f.rw);
    }
  }

  // 6. corrections by recomputation in binary64
  for (int t = warp; t < nc; t += nwarps) {
    if (how[t] == -2) continue;
    const CandEntry ce = cand[sidx[t]];
    const int p = A.kp(keys[t]);
    const Geo G = A.geo(p);
    const int64_t r = A.kr(keys[t]), c = A.kc(keys[t]);
    if (how[t] == -1) {
      if (lane == 0)
        push_report(report, cnt, p, (int32_t)r, (int32_t)c, ABFT_KIND_UNCORRECTABLE, ce.side, 0.0,
                    ce.re, ce.rw);
      continue;
    }
    double s = 0.0, expect;
    if (how[t] == 0) {
      const int64_t I = r / G.vb_r, i0 = I * G.vb_r, i1 = min(i0 + G.vb_r, G.m);
      for (int64_t i = i0 + lane; i < i1; i += 32)
        if (i != r) s += A.ldc(p, i, c);
      expect = A.expect_col(p, I, c);
    } else {
      const int64_t J = c / G.vb_c, j0 = J * G.vb_c, j1 = min(j0 + G.vb_c, G.n);
      for (int64_t j = j0 + lane; j < j1; j += 32)
        if (j != c) s += A.ldc(p, r, j);
      expect = A.expect_row(p, r, J);
    }
    s = warp_sum(s);
    if (lane == 0) {
      const double delta = A.stc(p, r, c, expect - s);
      push_report(report, cnt, p, (int32_t)r, (int32_t)c, mkind[t], ce.side, delta, ce.re, ce.rw);
    }
  }
  __syncthreads();

  // 7. re-check both lines of every corrected element (each line once)
  for (int t = warp; t < nc; t += nwarps) {
    if (how[t] < 0) continue;
    const int p = A.kp(keys[t]);
    const Geo G = A.geo(p);
    const int32_t r = A.kr(keys[t]), c = A.kc(keys[t]);
    const int64_t I = r / G.vb_r, J = c / G.vb_c;
    bool dup_c = false, dup_r = false;
    for (int u = 0; u < t; ++u) {
      if (how[u] < 0 || A.kp(keys[u]) != p) continue;
      const int32_t r2 = A.kr(keys[u]), c2 = A.kc(keys[u]);
      if (c2 == c && r2 / G.vb_r == I) dup_c = true;
      if (r2 == r && c2 / G.vb_c == J) dup_r = true;
    }
    double re, rw;
    if (!dup_c && A.recheck_col(p, I, c, re, rw) && lane == 0)  // warp-wide
      push_report(report, cnt, p, -1, c, ABFT_KIND_UNCORRECTABLE, 0, 0.0, re, rw);
    if (!dup_r && A.recheck_row(p, r, J, re, rw))
      push_report(report, cnt, p, r, -1, ABFT_KIND_UNCORRECTABLE, 1, 0.0, re, rw);
  }
}

template <typename TC>
__global__ void __launch_bounds__(kLocThreads, 1) k_locate_correct(const CheckArgs a) {
  if (a.timeout && *a.timeout) return;  // an incomplete product: write nothing
  const SinglePol<TC> A{a};
  locate_body(A, a.cnt, a.colf, a.rowf, a.cand, a.report);
}

// ---------------- grouped verify (fused observed sums, many problems)

__device__ __forceinline__ void grp_col_taus(const GProb& P, double s, int64_t I, int64_t j,
                                             double& te, double& tw) {
  const double nb = P.nBcol[j];
  te = s * nb * (P.f1c * P.nAblk[4 * I + 0] + P.f2 * P.nAblk[4 * I + 2]);
  tw = s * nb * (P.f1c * P.nAblk[4 * I + 1] + P.f2 * P.nAblk[4 * I + 3]);
}
__device__ __forceinline__ void grp_row_taus(const GProb& P, double s, int64_t i, int64_t J,
                                             double& te, double& tw) {
  const double na = P.nArow[i];
  te = s * na * (P.f1r * P.nBblk[4 * J + 0] + P.f2 * P.nBblk[4 * J + 2]);
  tw = s * na * (P.f1r * P.nBblk[4 * J + 1] + P.f2 * P.nBblk[4 * J + 3]);
}
// Expected sums: the products of the hi and lo checksum pieces, added in binary64.
__device__ __forceinline__ double grp_expect_col(const GProb& P, int64_t I, int64_t j, int w) {
  return (double)P.E16[(4 * I + 2 * w) * P.n + j] + (double)P.E16[(4 * I + 2 * w + 1) * P.n + j];
}
__device__ __forceinline__ double grp_expect_row(const GProb& P, int64_t i, int64_t J, int w) {
  return (double)P.F16[i * P.C16 + 4 * J + 2 * w] + (double)P.F16[i * P.C16 + 4 * J + 2 * w + 1];
}

struct GroupPol {
  const GProb* probs;
  double s;
  __device__ __forceinline__ Geo geo(int p) const {
    return Geo{probs[p].m, probs[p].n, kGrpVbR, kGrpVbC, kGrpEr, kGrpEc};
  }
  __device__ __forceinline__ double ldc(int p, int64_t i, int64_t j) const {
    return (double)probs[p].C[i * probs[p].ldc + j];
  }
  __device__ __forceinline__ double stc(int p, int64_t i, int64_t j, double v) const {
    float* c = probs[p].C + i * probs[p].ldc + j;
    const float old = *c, nv = (float)v;
    *c = nv;
    return (double)old - (double)nv;
  }
  __device__ __forceinline__ double expect_col(int p, int64_t I, int64_t j) const {
    return grp_expect_col(probs[p], I, j, 0);
  }
  __device__ __forceinline__ double tau_col(int p, int64_t I, int64_t j) const {
    double te, tw;
    grp_col_taus(probs[p], s, I, j, te, tw);
    return te;
  }
  __device__ __forceinline__ double tau_row(int p, int64_t i, int64_t J) const {
    double te, tw;
    grp_row_taus(probs[p], s, i, J, te, tw);
    return te;
  }
  __device__ __forceinline__ double expect_row(int p, int64_t i, int64_t J) const {
    return grp_expect_row(probs[p], i, J, 0);
  }
  // Column line re-read from C (binary32 sums, as the product's epilogue),
  // warp-wide (lanes split the rows); the result is valid in every lane.
  __device__ __forceinline__ bool recheck_col(int p, int64_t I, int64_t j, double& re,
                                              double& rw) const {
    const GProb& P = probs[p];
    const int lane = threadIdx.x & 31;
    const int64_t i0 = I * kGrpVbR, i1 = min(i0 + (int64_t)kGrpVbR, P.m);
    const float sc = scalbnf(1.0f, -kGrpEr);
    float se = 0.f, sw = 0.f;
    for (int64_t i = i0 + lane; i < i1; i += 32) {
      const float x = P.C[i * P.ldc + j];
      se += x;
      sw = fmaf((float)(i - i0 + 1) * sc, x, sw);
    }
    se = warp_sum_t<float>(se);
    sw = warp_sum_t<float>(sw);
    re = (double)se - grp_expect_col(P, I, j, 0);
    rw = (double)sw - grp_expect_col(P, I, j, 1);
    double te, tw;
    grp_col_taus(P, s, I, j, te, tw);
    return is_flagged(re, rw, te, tw);
  }
  // Warp-wide; the result is valid in lane 0.
  __device__ __forceinline__ bool recheck_row(int p, int64_t i, int64_t J, double& re,
                                              double& rw) const {
    const GProb& P = probs[p];
    const int lane = threadIdx.x & 31;
    const int64_t j0 = J * kGrpVbC, j1 = min(j0 + (int64_t)kGrpVbC, P.n);
    const float sc = scalbnf(1.0f, -kGrpEc);
    float se = 0.f, sw = 0.f;
    for (int64_t j = j0 + lane; j < j1; j += 32) {
      const float x = P.C[i * P.ldc + j];
      se += x;
      sw = fmaf((float)(j - j0 + 1) * sc, x, sw);
    }
    se = warp_sum_t<float>(se);
    sw = warp_sum_t<float>(sw);
    re = (double)se - grp_expect_row(P, i, J, 0);
    rw = (double)sw - grp_expect_row(P, i, J, 1);
    double te, tw;
    grp_row_taus(P, s, i, J, te, tw);
    return lane == 0 && is_flagged(re, rw, te, tw);
  }
  // problem (23 bits) | row (20) | column (20) | side
  __device__ __forceinline__ uint64_t key(int p, int64_t r, int64_t c, int side) const {
    return ((uint64_t)p << 41) | ((uint64_t)r << 21) | ((uint64_t)c << 1) | (uint64_t)side;
  }
  __device__ __forceinline__ int kp(uint64_t k) const { return (int)(k >> 41); }
  __device__ __forceinline__ int32_t kr(uint64_t k) const { return (int32_t)((k >> 21) & 0xFFFFFu); }
  __device__ __forceinline__ int32_t kc(uint64_t k) const { return (int32_t)((k >> 1) & 0xFFFFFu); }
};

// The verify screen.  A line passes when, evaluated in fp32, both residuals
// are within 0.9 of their thresholds; any other line is evaluated in binary64
// and flagged by the binary64 rule.  The fp32 evaluation differs from the
// binary64 one by at most u32 (|expected| + |r|) plus a few u32 of the
// threshold, and |expected| <= ||checksum row|| ||B_:j|| <= tau / (s f2) with
// s f2 >= 4 * 2^-17, so u32 |expected| <= 2^-9 tau: a line the screen passes
// is never one the binary64 rule flags (and non-finite sums never pass).
__device__ __forceinline__ bool screen_pass(float se, float sw, float ee, float ew, float te,
                                            float tw) {
  const float re = se - ee, rw = sw - ew;
  return fabsf(re) <= 0.9f * te && fabsf(rw) <= 0.9f * tw;  // false for NaN
}

// Column lines (problem, verify block I, column j) from the observed column
// sums of the product's epilogue (verify block = tile row).  CTA = 256 columns
// of one verify block, kGrpColThreads threads of 4 columns each: every load of
// a thread (the four 32-row blocks of observed sums, the four checksum
// pieces, the column norms) is issued before the first sum, as 16-byte loads
// when the rows are 16-byte aligned (n a multiple of 4; the workspace regions
// are 256-byte aligned).
constexpr int kGrpColThreads = 64;
__device__ __forceinline__ void ld4(const float* p, bool vec, int nv, float (&v)[4]) {
  if (vec) {
    const float4 x = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = u < nv ? __ldg(p + u) : 0.f;
  }
}
__global__ void __launch_bounds__(kGrpColThreads) k_grp_col(const GProb* __restrict__ probs,
                                                            const int2* __restrict__ tab,
                                                            double s, int32_t* cnt,
                                                            FlagEntry* colf) {
  const int2 e = tab[blockIdx.x];
  const int p = e.x;
  const GProb& P = probs[p];
  const int64_t n = P.n, ncx = cdiv(n, 256);
  const int64_t I = e.y / ncx, j0 = (e.y % ncx) * 256 + 4 * threadIdx.x;
  if (j0 >= n) return;
  const int nv = (int)min((int64_t)4, n - j0);  // columns of this thread
  const bool vec = (n & 3) == 0;                // then nv == 4 and every row is aligned
  // the verify block (one tile row) is four 32-row blocks of observed sums
  const int64_t nb32 = cdiv(P.m, 32);
  float pe[4][4], pw[4][4], ex[4][4], nb[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t b = 4 * I + q;
    if (b < nb32) {
      ld4(P.obs_col + (b * 2 + 0) * n + j0, vec, nv, pe[q]);
      ld4(P.obs_col + (b * 2 + 1) * n + j0, vec, nv, pw[q]);
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) pe[q][u] = pw[q][u] = 0.f;
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) ld4(P.E16 + (4 * I + r) * n + j0, vec, nv, ex[r]);
  ld4(P.nBcol32 + j0, vec, nv, nb);
  const float ta = P.tauA[2 * I], tw32 = P.tauA[2 * I + 1];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    if (u >= nv) break;
    const int64_t j = j0 + u;
    const float se32 = ((pe[0][u] + pe[1][u]) + pe[2][u]) + pe[3][u];
    const float sw32 = ((pw[0][u] + pw[1][u]) + pw[2][u]) + pw[3][u];
    if (screen_pass(se32, sw32, ex[0][u] + ex[1][u], ex[2][u] + ex[3][u], nb[u] * ta,
                    nb[u] * tw32))
      continue;
    const double se = (double)se32, sw = (double)sw32;
    const int nf = (isfinite(se) && isfinite(sw)) ? 0 : 1;
    const double re = se - grp_expect_col(P, I, j, 0), rw = sw - grp_expect_col(P, I, j, 1);
    double te, tw;
    grp_col_taus(P, s, I, j, te, tw);
    if (nf == 0 && !is_flagged(re, rw, te, tw)) continue;
    const int slot = atomicAdd(&cnt[kCntColFlags], 1);
    if (slot < kCapFlags) colf[slot] = FlagEntry{(int32_t)I, (int32_t)j, nf, p, re, rw};
  }
}

// Row lines (problem, row i, verify block J) from the observed row sums over
// column groups.  Each thread takes kGrpRowLines consecutive lines of the
// problem's (row, verify block) order (one division for the first, the rest by
// increment); with the grouped column groups (g = 128, two per verify block)
// every load of the thread is issued before the first sum.
__device__ __forceinline__ void grp_row_line(const GProb& P, int p, double s, int64_t i,
                                             int64_t J, float se32, float sw32, float4 F,
                                             float na, float2 tb, int32_t* cnt,
                                             FlagEntry* rowf) {
  if (screen_pass(se32, sw32, F.x + F.y, F.z + F.w, na * tb.x, na * tb.y)) return;
  const int64_t j0 = J * kGrpVbC, j1 = min(j0 + (int64_t)kGrpVbC, P.n);
  const int64_t g0 = j0 / P.g, g1 = min(cdiv(j1, P.g), P.ngrp);
  double se = 0.0, sw = 0.0;
  for (int64_t gr = g0; gr < g1; ++gr) {
    se += (double)P.obs_row[(i * P.ngrp + gr) * 2 + 0];
    sw += (double)P.obs_row[(i * P.ngrp + gr) * 2 + 1];
  }
  const int nf = (isfinite(se) && isfinite(sw)) ? 0 : 1;
  const double re = se - grp_expect_row(P, i, J, 0), rw = sw - grp_expect_row(P, i, J, 1);
  double te, tw;
  grp_row_taus(P, s, i, J, te, tw);
  if (nf == 0 && !is_flagged(re, rw, te, tw)) return;
  const int slot = atomicAdd(&cnt[kCntRowFlags], 1);
  if (slot < kCapFlags) rowf[slot] = FlagEntry{(int32_t)i, (int32_t)J, nf, p, re, rw};
}
__global__ void __launch_bounds__(kThreads) k_grp_row(const GProb* __restrict__ probs,
                                                      const int2* __restrict__ tab, double s,
                                                      int32_t* cnt, FlagEntry* rowf) {
  const int2 e = tab[blockIdx.x];
  const int p = e.x;
  const GProb& P = probs[p];
  const int64_t nvc = P.nvc, nlines = P.m * nvc;
  const int64_t t0 = ((int64_t)e.y * kThreads + threadIdx.x) * kGrpRowLines;
  if (t0 >= nlines) return;
  const int nl = (int)min((int64_t)kGrpRowLines, nlines - t0);
  int64_t i[kGrpRowLines], J[kGrpRowLines];
  i[0] = t0 / nvc;
  J[0] = t0 - i[0] * nvc;
#pragma unroll
  for (int u = 1; u < kGrpRowLines; ++u) {
    const bool wrap = J[u - 1] + 1 == nvc;
    i[u] = wrap ? i[u - 1] + 1 : i[u - 1];
    J[u] = wrap ? 0 : J[u - 1] + 1;
  }
  if (2 * P.g == kGrpVbC) {
    float4 F[kGrpRowLines];
    float2 a[kGrpRowLines], b[kGrpRowLines], tb[kGrpRowLines];
    float na[kGrpRowLines];
    bool two[kGrpRowLines];
#pragma unroll
    for (int u = 0; u < kGrpRowLines; ++u) {
      if (u >= nl) break;
      // F16 row i, pieces 4J .. 4J + 3 (C16 = 4 nvc: 16-byte aligned); the
      // (e, w) pairs of the line's one or two column groups (8-byte aligned)
      F[u] = __ldg(reinterpret_cast<const float4*>(P.F16 + i[u] * P.C16 + 4 * J[u]));
      na[u] = __ldg(P.nArow32 + i[u]);
      tb[u] = __ldg(reinterpret_cast<const float2*>(P.tauB + 2 * J[u]));
      const float* orow = P.obs_row + (i[u] * P.ngrp + 2 * J[u]) * 2;
      two[u] = 2 * J[u] + 1 < P.ngrp;
      a[u] = __ldg(reinterpret_cast<const float2*>(orow));
      b[u] = two[u] ? __ldg(reinterpret_cast<const float2*>(orow + 2)) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < kGrpRowLines; ++u) {
      if (u >= nl) break;
      float se32 = 0.f + a[u].x, sw32 = 0.f + a[u].y;
      if (two[u]) {
        se32 += b[u].x;
        sw32 += b[u].y;
      }
      grp_row_line(P, p, s, i[u], J[u], se32, sw32, F[u], na[u], tb[u], cnt, rowf);
    }
  } else {
    for (int u = 0; u < nl; ++u) {
      const int64_t j0 = J[u] * kGrpVbC, j1 = min(j0 + (int64_t)kGrpVbC, P.n);
      const int64_t g0 = j0 / P.g, g1 = min(cdiv(j1, P.g), P.ngrp);
      float se32 = 0.f, sw32 = 0.f;
      for (int64_t gr = g0; gr < g1; ++gr) {
        se32 += P.obs_row[(i[u] * P.ngrp + gr) * 2 + 0];
        sw32 += P.obs_row[(i[u] * P.ngrp + gr) * 2 + 1];
      }
      grp_row_line(P, p, s, i[u], J[u], se32, sw32,
                   *reinterpret_cast<const float4*>(P.F16 + i[u] * P.C16 + 4 * J[u]),
                   P.nArow32[i[u]], *reinterpret_cast<const float2*>(P.tauB + 2 * J[u]), cnt,
                   rowf);
    }
  }
}

__global__ void __launch_bounds__(kLocThreads, 1) k_grp_locate(const GProb* probs, double s,
                                                               int32_t* cnt, const FlagEntry* colf,
                                                               const FlagEntry* rowf,
                                                               CandEntry* cand,
                                                               abft_fault* report) {
  if (cnt[kCntTimeout]) return;  // the group's product timed out: write nothing
  const GroupPol A{probs, s};
  locate_body(A, cnt, colf, rowf, cand, report);
}

// Erased blocks rows[0..t) of block column bj (t <= kMaxBlockChecksums): for
// every element position (r, j) of the column's blocks,
//   rhs_l = S^(l)[r][j] - sum_{I not erased} c_{l,I} C[I*bs + r][j],   l < t,
//   C[rows[u]*bs + r][j] = sum_l minv[u][l] rhs_l,
// all in binary64 (t = 1: the block checksum minus the sum of the survivors).
// Grid (ceil(bc/256), bs).
struct RecoverSet {
  int t;
  int rows[kMaxBlockChecksums];
  double minv[kMaxBlockChecksums * kMaxBlockChecksums];
};

template <typename TC>
__global__ void __launch_bounds__(kThreads) k_recover(TC* C, int64_t ldc, const double* S,
                                                      int64_t n, int p, int64_t bs, int64_t bc,
                                                      int bj, const RecoverSet rs,
                                                      const int32_t* timeout) {
  const int64_t jj = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (jj >= bc) return;
  if (timeout && *timeout) return;  // block checksums of an incomplete product
  const int64_t j = (int64_t)bj * bc + jj;
  int e = 0;
  while ((1 << e) <= p) ++e;
  for (int64_t r = blockIdx.y; r < bs; r += gridDim.y) {
    double sum[kMaxBlockChecksums] = {0.0, 0.0, 0.0, 0.0};
    for (int I = 0; I < p; ++I) {
      bool erased = false;
#pragma unroll
      for (int u = 0; u < kMaxBlockChecksums; ++u) erased |= u < rs.t && rs.rows[u] == I;
      if (erased) continue;
      const double v = (double)C[(I * bs + r) * ldc + j];
      const double x = ldexp((double)(2 * I + 1 - p), -e);
      double c = 1.0;  // c_{l,I} = x^l
#pragma unroll
      for (int l = 0; l < kMaxBlockChecksums; ++l) {
        if (l < rs.t) sum[l] += c * v;
        c *= x;
      }
    }
    double rhs[kMaxBlockChecksums];
#pragma unroll
    for (int l = 0; l < kMaxBlockChecksums; ++l)
      rhs[l] = l < rs.t ? S[(l * bs + r) * n + j] - sum[l] : 0.0;
#pragma unroll
    for (int u = 0; u < kMaxBlockChecksums; ++u) {
      if (u >= rs.t) break;
      double xu = 0.0;
#pragma unroll
      for (int l = 0; l < kMaxBlockChecksums; ++l)
        if (l < rs.t) xu += rs.minv[u * rs.t + l] * rhs[l];
      C[((int64_t)rs.rows[u] * bs + r) * ldc + j] = (TC)xu;
    }
  }
}

// One rank's share of the rebuild of a block of block column bj when the
// block rows are spread over several GPUs (section 3.3: the lost block is the
// block checksum minus the sum of the survivors, formed by one reduction over
// the processes of the block column).  out[r][jj] (bs x bc, binary64):
//   (S == nullptr ? 0 : S[r][j]) - sum over local block rows I != skip of C[I bs + r][j],
// j = bj bc + jj.  The sum of every rank's share is the lost block.  Grid
// (ceil(bc/256), min(bs, 65535)).
template <typename TC>
__global__ void __launch_bounds__(kThreads) k_block_partial(const TC* C, int64_t ldc,
                                                            const double* S, int64_t n, int p,
                                                            int64_t bs, int64_t bc, int bj,
                                                            int skip, double* out) {
  const int64_t jj = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (jj >= bc) return;
  const int64_t j = (int64_t)bj * bc + jj;
  for (int64_t r = blockIdx.y; r < bs; r += gridDim.y) {
    double sum = 0.0;
    for (int I = 0; I < p; ++I)
      if (I != skip) sum += (double)C[(I * bs + r) * ldc + j];
    out[r * bc + jj] = (S ? S[r * n + j] : 0.0) - sum;
  }
}

// The rebuilt block written into C (rounded to C's type): C[bi bs + r][bj bc + jj]
// = src[r][jj].  Grid (ceil(bc/256), min(bs, 65535)).
template <typename TC>
__global__ void __launch_bounds__(kThreads) k_block_store(TC* C, int64_t ldc, const double* src,
                                                          int64_t bs, int64_t bc, int bi, int bj,
                                                          const int32_t* timeout) {
  const int64_t jj = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (jj >= bc) return;
  if (timeout && *timeout) return;  // checksums of an incomplete product
  for (int64_t r = blockIdx.y; r < bs; r += gridDim.y)
    C[((int64_t)bi * bs + r) * ldc + (int64_t)bj * bc + jj] = (TC)src[r * bc + jj];
}

struct Flip {
  int64_t row, col;
  int32_t bit, pad;
};
struct FlipList {
  int32_t n, pad;
  Flip f[64];
};

template <typename TC, typename TU>
__global__ void k_inject(TC* C, int64_t ldc, const FlipList fl) {
  const int t = threadIdx.x;
  if (t >= fl.n) return;
  TU* u = reinterpret_cast<TU*>(C + fl.f[t].row * ldc + fl.f[t].col);
  *u ^= (TU)1 << fl.f[t].bit;
}

template <typename TC>
__global__ void k_erase(TC* C, int64_t ldc, int64_t r0, int64_t c0, int64_t bs, int64_t bc) {
  const int64_t jj = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (jj >= bc) return;
  for (int64_t t = blockIdx.y; t < bs; t += gridDim.y) C[(r0 + t) * ldc + c0 + jj] = (TC)nan("");
}

unsigned gy(int64_t v) { return (unsigned)(v < 65535 ? v : 65535); }

CheckArgs make_args(const Plan& P, void* C, void* ws) {
  char* w = static_cast<char*>(ws);
  Scratch S = scratch_view(P, ws);
  CheckArgs a{};
  a.C = C;
  a.ldc = P.d.ldc; a.m = P.d.m; a.n = P.d.n;
  a.E = reinterpret_cast<const double*>(w + P.L.E);
  a.F = reinterpret_cast<const double*>(w + P.L.F);
  a.nArow = reinterpret_cast<const double*>(w + P.L.nArow);
  a.nAblk = reinterpret_cast<const double*>(w + P.L.nAblk);
  a.nBcol = reinterpret_cast<const double*>(w + P.L.nBcol);
  a.nBblk = reinterpret_cast<const double*>(w + P.L.nBblk);
  a.carA = reinterpret_cast<const double*>(w + P.L.car_a);
  a.carB = reinterpret_cast<const double*>(w + P.L.car_b);
  a.vb_r = P.d.vb_rows; a.vb_c = P.d.vb_cols; a.er = P.er; a.ec = P.ec;
  a.nvr = P.nvr; a.nvc = P.nvc; a.Cc = P.Cc; a.bs = P.bs; a.bc = P.bc;
  a.s = P.s; a.f1c = P.f1_col; a.f2c = P.f2_col; a.f1r = P.f1_row; a.f2r = P.f2_row;
  a.colf = S.colf; a.rowf = S.rowf; a.cnt = S.cnt; a.report = S.report; a.cand = S.cand;
  a.timeout = P.d.dtype == ABFT_F64 ? nullptr : S.cnt + kCntTimeout;
  return a;
}

template <typename TC>
cudaError_t verify_t(const Plan& P, void* C, void* ws, const Erased& er, bool reread,
                     cudaStream_t st) {
  CheckArgs a = make_args(P, C, ws);
  a.erased = er;
  const int64_t m = P.d.m, n = P.d.n;
  if (reread) {
    k_col_check<TC><<<dim3((unsigned)cdiv(n, kThreads), gy(P.nvr)), kThreads, 0, st>>>(
        a, 0, n, 0, P.nvr, 0);
    k_row_check<TC><<<(unsigned)cdiv(m * P.nvc * 32, kThreads), kThreads, 0, st>>>(a);
  } else {
    const char* w = static_cast<const char*>(ws);
    k_col_fused<<<dim3((unsigned)cdiv(n, kThreads), gy(P.nvr)), kThreads, 0, st>>>(
        a, reinterpret_cast<const float*>(w + P.L.obs_col), P.ntr_obs);
    k_row_fused<<<(unsigned)cdiv(m * P.nvc, kThreads), kThreads, 0, st>>>(
        a, reinterpret_cast<const float*>(w + P.L.obs_row), P.g, P.ngrp);
  }
  k_locate_correct<TC><<<1, kLocThreads, 0, st>>>(a);
  count_launches(3);
  return cudaGetLastError();
}

template <typename TC>
cudaError_t recover_t(const Plan& P, void* C, void* ws, int bj, const int* rows, int t,
                      const double* minv, cudaStream_t st) {
  CheckArgs a = make_args(P, C, ws);
  const double* S = a.E + 2 * P.nvr * P.d.n;
  RecoverSet rs{};
  rs.t = t;
  for (int u = 0; u < t; ++u) rs.rows[u] = rows[u];
  for (int x = 0; x < t * t; ++x) rs.minv[x] = minv[x];
  k_recover<TC><<<dim3((unsigned)cdiv(P.bc, kThreads), gy(P.bs)), kThreads, 0, st>>>(
      static_cast<TC*>(C), P.d.ldc, S, P.d.n, P.d.grid_p, P.bs, P.bc, bj, rs, a.timeout);
  for (int u = 0; u < t; ++u) {  // re-check the rebuilt blocks' column lines
    const int64_t I0 = ((int64_t)rows[u] * P.bs) / P.d.vb_rows;
    const int64_t I1 = cdiv(((int64_t)rows[u] + 1) * P.bs, P.d.vb_rows);
    k_col_check<TC><<<dim3((unsigned)cdiv(P.bc, kThreads), gy(I1 - I0)), kThreads, 0, st>>>(
        a, (int64_t)bj * P.bc, ((int64_t)bj + 1) * P.bc, I0, I1, 1);
  }
  count_launches(1 + t);
  return cudaGetLastError();
}

template <typename TC>
cudaError_t block_partial_t(const Plan& P, const void* C, const void* ws, int skip, int bj,
                            bool with_checksum, double* out, cudaStream_t st) {
  const char* w = static_cast<const char*>(ws);
  const double* S = with_checksum ? reinterpret_cast<const double*>(w + P.L.E) + 2 * P.nvr * P.d.n
                                  : nullptr;
  k_block_partial<TC><<<dim3((unsigned)cdiv(P.bc, kThreads), gy(P.bs)), kThreads, 0, st>>>(
      static_cast<const TC*>(C), P.d.ldc, S, P.d.n, P.d.grid_p, P.bs, P.bc, bj, skip, out);
  count_launches(1);
  return cudaGetLastError();
}

template <typename TC>
cudaError_t block_restore_t(const Plan& P, void* C, void* ws, int bi, int bj, const double* src,
                            cudaStream_t st) {
  CheckArgs a = make_args(P, C, ws);
  k_block_store<TC><<<dim3((unsigned)cdiv(P.bc, kThreads), gy(P.bs)), kThreads, 0, st>>>(
      static_cast<TC*>(C), P.d.ldc, src, P.bs, P.bc, bi, bj, a.timeout);
  const int64_t I0 = ((int64_t)bi * P.bs) / P.d.vb_rows;
  const int64_t I1 = cdiv(((int64_t)bi + 1) * P.bs, P.d.vb_rows);
  k_col_check<TC><<<dim3((unsigned)cdiv(P.bc, kThreads), gy(I1 - I0)), kThreads, 0, st>>>(
      a, (int64_t)bj * P.bc, ((int64_t)bj + 1) * P.bc, I0, I1, 1);
  count_launches(2);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_block_partial(const Plan& P, const void* C, const void* ws, int skip, int bj,
                                 bool with_checksum, double* out, cudaStream_t st) {
  return P.d.dtype == ABFT_F64 ? block_partial_t<double>(P, C, ws, skip, bj, with_checksum, out, st)
                               : block_partial_t<float>(P, C, ws, skip, bj, with_checksum, out, st);
}

cudaError_t launch_block_restore(const Plan& P, void* C, void* ws, int bi, int bj,
                                 const double* src, cudaStream_t st) {
  return P.d.dtype == ABFT_F64 ? block_restore_t<double>(P, C, ws, bi, bj, src, st)
                               : block_restore_t<float>(P, C, ws, bi, bj, src, st);
}

cudaError_t launch_verify(const Plan& P, void* C, void* ws, const Erased& er, bool reread,
                          cudaStream_t st) {
  return P.d.dtype == ABFT_F64 ? verify_t<double>(P, C, ws, er, true, st)
                               : verify_t<float>(P, C, ws, er, reread, st);
}

namespace {
struct InjList {
  int32_t n, first, total, last;
  InjectEntry e[64];
};
__global__ void k_set_inject(int32_t* hdr, const InjList L) {
  InjectEntry* ent = reinterpret_cast<InjectEntry*>(reinterpret_cast<char*>(hdr) + 16);
  const int t = threadIdx.x;
  if (t < L.n) ent[L.first + t] = L.e[t];
  if (L.last && t == 0) {
    hdr[1] = L.total;
    hdr[0] = kInjectMagic;
  }
}
}  // namespace

cudaError_t launch_set_inject_raw(int32_t* hdr, const InjectEntry* entries, int count,
                                  cudaStream_t st) {
  int t0 = 0;
  do {
    InjList L{};
    L.n = count - t0 < 64 ? count - t0 : 64;
    L.first = t0;
    L.total = count;
    L.last = t0 + L.n >= count;
    for (int t = 0; t < L.n; ++t) L.e[t] = entries[t0 + t];
    k_set_inject<<<1, 64, 0, st>>>(hdr, L);
    count_launches(1);
    t0 += L.n;
  } while (t0 < count);
  return cudaGetLastError();
}

cudaError_t launch_set_inject(const Plan& P, void* ws, const int64_t* rows, const int64_t* cols,
                              const int32_t* bits, int count, cudaStream_t st) {
  int32_t* hdr = reinterpret_cast<int32_t*>(static_cast<char*>(ws) + P.L.inject);
  InjectEntry e[kMaxInject];
  for (int t = 0; t < count && t < kMaxInject; ++t)
    e[t] = InjectEntry{(int32_t)rows[t], (int32_t)cols[t], bits[t], 0};
  return launch_set_inject_raw(hdr, e, count, st);
}

cudaError_t launch_recover(const Plan& P, void* C, void* ws, int bj, const int* rows, int t,
                           const double* minv, cudaStream_t st) {
  return P.d.dtype == ABFT_F64 ? recover_t<double>(P, C, ws, bj, rows, t, minv, st)
                               : recover_t<float>(P, C, ws, bj, rows, t, minv, st);
}

cudaError_t launch_inject(const Plan& P, void* C, const int64_t* rows, const int64_t* cols,
                          const int32_t* bits, int count, cudaStream_t st) {
  for (int t0 = 0; t0 < count; t0 += 64) {
    FlipList fl{};
    fl.n = count - t0 < 64 ? count - t0 : 64;
    for (int t = 0; t < fl.n; ++t) fl.f[t] = Flip{rows[t0 + t], cols[t0 + t], bits[t0 + t], 0};
    if (P.d.dtype == ABFT_F64)
      k_inject<double, unsigned long long><<<1, 64, 0, st>>>(static_cast<double*>(C), P.d.ldc, fl);
    else
      k_inject<float, unsigned int><<<1, 64, 0, st>>>(static_cast<float*>(C), P.d.ldc, fl);
    count_launches(1);
  }
  return cudaGetLastError();
}

cudaError_t launch_erase(const Plan& P, void* C, int bi, int bj, cudaStream_t st) {
  const dim3 grid((unsigned)cdiv(P.bc, kThreads), gy(P.bs));
  if (P.d.dtype == ABFT_F64)
    k_erase<double><<<grid, kThreads, 0, st>>>(static_cast<double*>(C), P.d.ldc,
                                               (int64_t)bi * P.bs, (int64_t)bj * P.bc, P.bs, P.bc);
  else
    k_erase<float><<<grid, kThreads, 0, st>>>(static_cast<float*>(C), P.d.ldc, (int64_t)bi * P.bs,
                                              (int64_t)bj * P.bc, P.bs, P.bc);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_group_verify(const GroupDev& G, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(G.cnt, 0, sizeof(int32_t) * kNumCleared, st);
  if (e != cudaSuccess || G.count == 0) return e;
  if (G.nctas[kGkColCheck] > 0)
    k_grp_col<<<(unsigned)G.nctas[kGkColCheck], kGrpColThreads, 0, st>>>(
        G.probs, G.tab[kGkColCheck], G.s, G.cnt, G.colf);
  if (G.nctas[kGkRowCheck] > 0)
    k_grp_row<<<(unsigned)G.nctas[kGkRowCheck], kThreads, 0, st>>>(
        G.probs, G.tab[kGkRowCheck], G.s, G.cnt, G.rowf);
  k_grp_locate<<<1, kLocThreads, 0, st>>>(G.probs, G.s, G.cnt, G.colf, G.rowf, G.cand, G.report);
  count_launches(3);
  return cudaGetLastError();
}

}  // namespace abft
