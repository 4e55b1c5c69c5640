// Checksum encoding for binary64 operands (section 2.1; the encoded operands
// of Eq. (1)).  All kernels stream A or B once per quantity with coalesced
// loads; reductions along the long dimension are two-stage (per-chunk
// partials, then an ordered sum) so the result does not depend on scheduling.

#include "internal.cuh"

namespace abft {
namespace {

constexpr int kThreads = 256;
constexpr int kRowsPerWarpB = 64;  // rows of B per warp in the row-checksum pass

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of v over the 256 threads of the block; valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < kThreads / 32; ++q) t += sh[q];
  return t;
}

// Column checksums of A per verify block: acs[2I] = e^T A_I, acs[2I+1] =
// w^T A_I, plus per-chunk partials of ||e^T A_I||^2 and ||w^T A_I||^2 at
// part[(2I + c) * nch + chunk].  Grid (ceil(k/256), <= 65535); thread = one
// column l of A.
__global__ void __launch_bounds__(kThreads) k_encA_cols(const double* __restrict__ A, int64_t lda,
                                                        int64_t m, int64_t k, int vb, int e,
                                                        double* __restrict__ acs,
                                                        double* __restrict__ part, int nch) {
  __shared__ double sh[kThreads / 32];
  const int64_t l = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const int64_t nvb = cdiv(m, vb);
  const double sc = scalbn(1.0, -e);
  for (int64_t I = blockIdx.y; I < nvb; I += gridDim.y) {
    const int64_t i0 = I * vb, i1 = min(i0 + (int64_t)vb, m);
    double se = 0.0, sw = 0.0;
    if (l < k) {
      const double* p = A + i0 * lda + l;
#pragma unroll 4
      for (int64_t i = i0; i < i1; ++i) {
        const double a = p[(i - i0) * lda];
        se += a;
        sw = fma((double)(i - i0 + 1) * sc, a, sw);
      }
      acs[(2 * I) * k + l] = se;
      acs[(2 * I + 1) * k + l] = sw;
    }
    const double q[2] = {se * se, sw * sw};
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const double t = block_sum(q[c], sh);
      if (threadIdx.x == 0) part[(2 * I + c) * nch + blockIdx.x] = t;
    }
  }
}

// Block checksum rows S_A[t] = sum_I A[I*bs + t] (erasure grid).
// Grid (ceil(k/256), bs).
__global__ void __launch_bounds__(kThreads) k_encA_block(const double* __restrict__ A, int64_t lda,
                                                         int64_t k, int p, int64_t bs, int f,
                                                         double* __restrict__ S) {
  const int64_t l = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (l >= k) return;
  // row c*bs + t of S: sum_I c_{c,I} A[I*bs + t] (block checksum c of the grid)
  for (int64_t ct = blockIdx.y; ct < f * bs; ct += gridDim.y) {
    const int c = (int)(ct / bs);
    const int64_t t = ct - c * bs;
    double s = 0.0;
    for (int I = 0; I < p; ++I) s += block_coef(c, I, p) * A[(I * bs + t) * lda + l];
    S[ct * k + l] = s;
  }
}

// ||A_{i,:}||_2, one warp per row.
__global__ void __launch_bounds__(kThreads) k_row_norms(const double* __restrict__ A, int64_t lda,
                                                        int64_t m, int64_t k,
                                                        double* __restrict__ out) {
  const int64_t i = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= m) return;
  double s = 0.0;
  for (int64_t l = lane; l < k; l += 32) {
    const double a = A[i * lda + l];
    s = fma(a, a, s);
  }
  s = warp_sum(s);
  if (lane == 0) out[i] = sqrt(s);
}

// Row checksums of B per verify block: bcs[l][2J] = B_J e, bcs[l][2J+1] = B_J w,
// plus per-chunk partials of ||B_J e||^2 and ||B_J w||^2 at
// part[(2J + c) * nch + chunk].  One warp per (J, chunk of 64 rows of B).
__global__ void __launch_bounds__(kThreads) k_encB_rows(const double* __restrict__ B, int64_t ldb,
                                                        int64_t k, int64_t n, int vb, int e,
                                                        double* __restrict__ bcs, int64_t Cc,
                                                        double* __restrict__ part, int nch) {
  const int lane = threadIdx.x & 31;
  const int64_t chunk = (int64_t)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
  if (chunk >= nch) return;
  const int64_t nvb = cdiv(n, vb);
  const double sc = scalbn(1.0, -e);
  for (int64_t J = blockIdx.y; J < nvb; J += gridDim.y) {
    const int64_t j0 = J * vb, j1 = min(j0 + (int64_t)vb, n);
    const int64_t l0 = chunk * kRowsPerWarpB, l1 = min(l0 + kRowsPerWarpB, k);
    double q0 = 0.0, q1 = 0.0;
    for (int64_t l = l0; l < l1; ++l) {
      double se = 0.0, sw = 0.0;
      for (int64_t j = j0 + lane; j < j1; j += 32) {
        const double b = B[l * ldb + j];
        se += b;
        sw = fma((double)(j - j0 + 1) * sc, b, sw);
      }
      se = warp_sum(se);
      sw = warp_sum(sw);
      if (lane == 0) {
        bcs[l * Cc + 2 * J] = se;
        bcs[l * Cc + 2 * J + 1] = sw;
      }
      q0 = fma(se, se, q0);
      q1 = fma(sw, sw, q1);
    }
    if (lane == 0) {
      part[(2 * J + 0) * nch + chunk] = q0;
      part[(2 * J + 1) * nch + chunk] = q1;
    }
  }
}

// Per-chunk partial sums of B_lj^2 for the column norms.  Grid (ceil(n/256), nch).
__global__ void __launch_bounds__(kThreads) k_col_sq(const double* __restrict__ B, int64_t ldb,
                                                     int64_t k, int64_t n,
                                                     double* __restrict__ part) {
  const int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (j >= n) return;
  const int64_t nch = cdiv(k, kThreads);
  for (int64_t c = blockIdx.y; c < nch; c += gridDim.y) {
    const int64_t l0 = c * kThreads, l1 = min(l0 + kThreads, k);
    double s = 0.0;
#pragma unroll 4
    for (int64_t l = l0; l < l1; ++l) {
      const double b = B[l * ldb + j];
      s = fma(b, b, s);
    }
    part[c * n + j] = s;
  }
}

// out[o] = sqrt(sum_c part[o*so + c*sc]) in chunk order.
__global__ void k_sum_sqrt(const double* __restrict__ part, int64_t nout, int64_t nch, int64_t so,
                           int64_t sc, double* __restrict__ out) {
  const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= nout) return;
  double s = 0.0;
  for (int64_t c = 0; c < nch; ++c) s += part[o * so + c * sc];
  out[o] = sqrt(s);
}

// Threshold norms of every verify block from the per-line norms and the
// checksum partials: nblk[4I] = sqrt(sum_{t in I} nvec_t^2), nblk[4I+1] =
// sqrt(sum (w_t nvec_t)^2), nblk[4I+2], nblk[4I+3] = sqrt of the summed
// partials of the two checksum vectors.  One thread per verify block.
__global__ void k_finalize_blk(const double* __restrict__ nvec, int64_t len, int vb, int e,
                               const double* __restrict__ part, int64_t nch,
                               double* __restrict__ nblk) {
  const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nvb = cdiv(len, vb);
  if (I >= nvb) return;
  const double sc = scalbn(1.0, -e);
  const int64_t t0 = I * vb, t1 = min(t0 + (int64_t)vb, len);
  double f0 = 0.0, f1 = 0.0, q0 = 0.0, q1 = 0.0;
  for (int64_t t = t0; t < t1; ++t) {
    const double v = nvec[t], wv = (double)(t - t0 + 1) * sc * v;
    f0 = fma(v, v, f0);
    f1 = fma(wv, wv, f1);
  }
  for (int64_t c = 0; c < nch; ++c) {
    q0 += part[(2 * I) * nch + c];
    q1 += part[(2 * I + 1) * nch + c];
  }
  nblk[4 * I + 0] = sqrt(f0);
  nblk[4 * I + 1] = sqrt(f1);
  nblk[4 * I + 2] = sqrt(q0);
  nblk[4 * I + 3] = sqrt(q1);
}

// ---------------------------------------------------------------- chained calls
// A chained product (section 3.2: stacked calls do not recompute checksums)
// takes its encoded rows of A / columns of B from an earlier product's
// expected checksums; the kernels below form the norms of those carried
// vectors and the bound of their deviation from the stored operand.

// part[r * nch + chunk] = sum over the chunk's 256 columns of acs[r][l]^2, the
// layout k_encA_cols leaves for the checksum-row norms (r = 2I + c).
// Grid (nch, <= 65535).
__global__ void __launch_bounds__(kThreads) k_rows_sq(const double* __restrict__ acs, int64_t k,
                                                      int64_t rows, double* __restrict__ part,
                                                      int nch) {
  __shared__ double sh[kThreads / 32];
  const int64_t l = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  for (int64_t r = blockIdx.y; r < rows; r += gridDim.y) {
    const double v = l < k ? acs[r * k + l] : 0.0;
    const double t = block_sum(v * v, sh);
    if (threadIdx.x == 0) part[r * nch + blockIdx.x] = t;
  }
}

// part[c * nch + chunk] = sum over the chunk's kRowsPerWarpB rows of
// bcs[l][c]^2, the layout k_encB_rows leaves (c = 2J + w).  One thread per
// (c, chunk).
__global__ void __launch_bounds__(kThreads) k_cols_sq(const double* __restrict__ bcs, int64_t k,
                                                      int64_t Cc, double* __restrict__ part,
                                                      int nch) {
  const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (t >= Cc * nch) return;
  const int64_t c = t / nch, chunk = t - c * nch;
  const int64_t l0 = chunk * kRowsPerWarpB, l1 = min(l0 + (int64_t)kRowsPerWarpB, k);
  double q = 0.0;
  for (int64_t l = l0; l < l1; ++l) {
    const double b = bcs[l * Cc + c];
    q = fma(b, b, q);
  }
  part[c * nch + chunk] = q;
}

// Deviation bound of checksums carried out of an earlier product: its
// deviation per line stays within that product's unscaled threshold, so the
// largest one of verify block I is at most
//   car[2I+c] = max_t nvec[t] * (f1 * nblk[4I+c] + f2 * nblk[4I+2+c] + car_prev[2I+c]),
// nvec the earlier product's column norms of B (row side: row norms of A).
// One CTA.
__global__ void __launch_bounds__(kThreads) k_carry(const double* __restrict__ nvec, int64_t len,
                                                    const double* __restrict__ nblk,
                                                    const double* __restrict__ car_prev,
                                                    int64_t nvb, double f1, double f2,
                                                    double* __restrict__ car) {
  __shared__ double sh[kThreads / 32];
  __shared__ double s_mx;
  double mx = 0.0;
  for (int64_t t = threadIdx.x; t < len; t += kThreads) mx = fmax(mx, nvec[t]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) v = fmax(v, sh[w]);
    s_mx = v;
  }
  __syncthreads();
  mx = s_mx;
  for (int64_t x = threadIdx.x; x < 2 * nvb; x += kThreads) {
    const int64_t I = x >> 1, c = x & 1;
    car[x] = mx * (f1 * nblk[4 * I + c] + f2 * nblk[4 * I + 2 + c] + car_prev[x]);
  }
}

}  // namespace

namespace {

// The encode's launch sequence, with its per-chunk partial sums at `part`
// (the workspace scratch, or the static array of abft_encode_noalloc).
cudaError_t encode_f64_into(const Plan& P, const double* A, const double* B, void* ws,
                            double* part, cudaStream_t st) {
  const abft_desc& d = P.d;
  char* w = static_cast<char*>(ws);
  double* acs = reinterpret_cast<double*>(w + P.L.acs);
  double* bcs = reinterpret_cast<double*>(w + P.L.bcs);
  double* nArow = reinterpret_cast<double*>(w + P.L.nArow);
  double* nAblk = reinterpret_cast<double*>(w + P.L.nAblk);
  double* nBcol = reinterpret_cast<double*>(w + P.L.nBcol);
  double* nBblk = reinterpret_cast<double*>(w + P.L.nBblk);
  const int nchA = (int)cdiv(d.k, kThreads);
  const int nchB = (int)cdiv(d.k, kRowsPerWarpB);
  const int nchC = (int)cdiv(d.k, kThreads);
  double* partA = part;
  double* partB = partA + 4 * P.nvr * nchA;
  double* partC = partB + 4 * P.nvc * nchB;

  auto gy = [](int64_t v) { return (unsigned)(v < 65535 ? v : 65535); };
  if (d.k == 0) {  // empty inner dimension: all checksums and norms are zero
    cudaMemsetAsync(nArow, 0, sizeof(double) * d.m, st);
    cudaMemsetAsync(nAblk, 0, sizeof(double) * 4 * P.nvr, st);
    cudaMemsetAsync(nBcol, 0, sizeof(double) * d.n, st);
    cudaMemsetAsync(nBblk, 0, sizeof(double) * 4 * P.nvc, st);
    return cudaGetLastError();
  }
  count_launches(P.bs > 0 ? 8 : 7);
  k_encA_cols<<<dim3((unsigned)nchA, gy(P.nvr)), kThreads, 0, st>>>(
      A, d.lda, d.m, d.k, d.vb_rows, P.er, acs, partA, nchA);
  if (P.bs > 0)
    k_encA_block<<<dim3((unsigned)cdiv(d.k, kThreads), gy(P.f * P.bs)), kThreads, 0, st>>>(
        A, d.lda, d.k, d.grid_p, P.bs, P.f, acs + 2 * P.nvr * d.k);
  k_row_norms<<<(unsigned)cdiv(d.m * 32, kThreads), kThreads, 0, st>>>(A, d.lda, d.m, d.k, nArow);
  k_encB_rows<<<dim3((unsigned)cdiv(nchB, kThreads / 32), gy(P.nvc)), kThreads, 0, st>>>(
      B, d.ldb, d.k, d.n, d.vb_cols, P.ec, bcs, P.Cc, partB, nchB);
  k_col_sq<<<dim3((unsigned)cdiv(d.n, kThreads), gy(nchC)), kThreads, 0, st>>>(
      B, d.ldb, d.k, d.n, partC);
  k_sum_sqrt<<<(unsigned)cdiv(d.n, 128), 128, 0, st>>>(partC, d.n, nchC, 1, d.n, nBcol);
  k_finalize_blk<<<(unsigned)cdiv(P.nvr, 128), 128, 0, st>>>(nArow, d.m, d.vb_rows, P.er, partA,
                                                             nchA, nAblk);
  k_finalize_blk<<<(unsigned)cdiv(P.nvc, 128), 128, 0, st>>>(nBcol, d.n, d.vb_cols, P.ec, partB,
                                                             nchB, nBblk);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_encode_f64(const Plan& P, const double* A, const double* B, void* ws,
                              cudaStream_t st) {
  return encode_f64_into(P, A, B, ws, scratch_view(P, ws).part, st);
}

// ---------------------------------------------------------------------------
// Encode without a workspace scratch region (abft_encode_noalloc).
//
// The encode's per-chunk partial sums normally live in the scratch part of the
// caller's workspace.  For callers that cannot allocate device memory, this
// variant keeps them in the file-scope array below instead.  The array is
// created by the CUDA runtime when this module is loaded on a device and stays
// resident on every device that loads the library until the process exits.
// Every call shares it; every slot a call reads is first written by the same
// call, so nothing needs clearing, but calls that overlap on the GPU race on
// it.
constexpr size_t kStaticEncodePartBytes = size_t(8) << 20;  // 8 MiB
static __device__ __align__(256) double g_encode_part[kStaticEncodePartBytes / sizeof(double)];

size_t static_encode_part_bytes() { return kStaticEncodePartBytes; }

// In host code the array's name is only a stand-in, not a device address:
// the address on the current device is looked up with cudaGetSymbolAddress on
// every call (it is not cached, so a device reset or a new context cannot
// leave a stale pointer behind).
cudaError_t launch_encode_f64_noalloc(const Plan& P, const double* A, const double* B, void* ws,
                                      cudaStream_t st) {
  void* part = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&part, g_encode_part);
  if (e != cudaSuccess) return e;
  return encode_f64_into(P, A, B, ws, static_cast<double*>(part), st);
}

// Deviation bounds of the checksums carried out of an earlier product PL
// (workspace wsL): its column checksum rows (one pair per row verify block)
// and its row checksum columns (one pair per column verify block).
cudaError_t launch_carry_rows(const Plan& PL, const void* wsL, double* car, cudaStream_t st) {
  const char* wl = static_cast<const char*>(wsL);
  k_carry<<<1, kThreads, 0, st>>>(reinterpret_cast<const double*>(wl + PL.L.nBcol), PL.d.n,
                                  reinterpret_cast<const double*>(wl + PL.L.nAblk),
                                  reinterpret_cast<const double*>(wl + PL.L.car_a), PL.nvr,
                                  PL.f1_col, PL.f2_col, car);
  return cudaGetLastError();
}
cudaError_t launch_carry_cols(const Plan& PR, const void* wsR, double* car, cudaStream_t st) {
  const char* wr = static_cast<const char*>(wsR);
  k_carry<<<1, kThreads, 0, st>>>(reinterpret_cast<const double*>(wr + PR.L.nArow), PR.d.m,
                                  reinterpret_cast<const double*>(wr + PR.L.nBblk),
                                  reinterpret_cast<const double*>(wr + PR.L.car_b), PR.nvc,
                                  PR.f1_row, PR.f2_row, car);
  return cudaGetLastError();
}

cudaError_t launch_encode_f64_chained(const Plan& P, const double* A, const double* B, void* ws,
                                      const Plan* PL, const void* wsL, const Plan* PR,
                                      const void* wsR, cudaStream_t st) {
  const abft_desc& d = P.d;
  if (d.k == 0) return launch_encode_f64(P, A, B, ws, st);  // nothing to carry: zero norms
  char* w = static_cast<char*>(ws);
  double* acs = reinterpret_cast<double*>(w + P.L.acs);
  double* bcs = reinterpret_cast<double*>(w + P.L.bcs);
  double* nArow = reinterpret_cast<double*>(w + P.L.nArow);
  double* nAblk = reinterpret_cast<double*>(w + P.L.nAblk);
  double* nBcol = reinterpret_cast<double*>(w + P.L.nBcol);
  double* nBblk = reinterpret_cast<double*>(w + P.L.nBblk);
  double* carA = reinterpret_cast<double*>(w + P.L.car_a);
  double* carB = reinterpret_cast<double*>(w + P.L.car_b);
  Scratch S = scratch_view(P, ws);
  const int nchA = (int)cdiv(d.k, kThreads);
  const int nchB = (int)cdiv(d.k, kRowsPerWarpB);
  const int nchC = (int)cdiv(d.k, kThreads);
  double* partA = S.part;
  double* partB = partA + 4 * P.nvr * nchA;
  double* partC = partB + 4 * P.nvc * nchB;
  auto gy = [](int64_t v) { return (unsigned)(v < 65535 ? v : 65535); };
  cudaError_t e = cudaSuccess;
  int launches = 0;

  if (PL) {  // rows of A: the earlier product's E (verify rows, then block checksum rows)
    const char* wl = static_cast<const char*>(wsL);
    const double* EL = reinterpret_cast<const double*>(wl + PL->L.E);
    e = cudaMemcpyAsync(acs, EL, sizeof(double) * (size_t)P.R * d.k, cudaMemcpyDeviceToDevice,
                        st);
    if (e != cudaSuccess) return e;
    k_rows_sq<<<dim3((unsigned)nchA, gy(2 * P.nvr)), kThreads, 0, st>>>(acs, d.k, 2 * P.nvr,
                                                                         partA, nchA);
    launch_carry_rows(*PL, wsL, carA, st);
    launches += 2;
  } else {
    k_encA_cols<<<dim3((unsigned)nchA, gy(P.nvr)), kThreads, 0, st>>>(
        A, d.lda, d.m, d.k, d.vb_rows, P.er, acs, partA, nchA);
    ++launches;
    if (P.bs > 0) {
      k_encA_block<<<dim3((unsigned)cdiv(d.k, kThreads), gy(P.f * P.bs)), kThreads, 0, st>>>(
          A, d.lda, d.k, d.grid_p, P.bs, P.f, acs + 2 * P.nvr * d.k);
      ++launches;
    }
  }
  k_row_norms<<<(unsigned)cdiv(d.m * 32, kThreads), kThreads, 0, st>>>(A, d.lda, d.m, d.k, nArow);

  if (PR) {  // columns of B: the earlier product's F (k x Cc)
    const char* wr = static_cast<const char*>(wsR);
    const double* FR = reinterpret_cast<const double*>(wr + PR->L.F);
    e = cudaMemcpyAsync(bcs, FR, sizeof(double) * (size_t)d.k * P.Cc, cudaMemcpyDeviceToDevice,
                        st);
    if (e != cudaSuccess) return e;
    k_cols_sq<<<(unsigned)cdiv(P.Cc * nchB, kThreads), kThreads, 0, st>>>(bcs, d.k, P.Cc, partB,
                                                                           nchB);
    launch_carry_cols(*PR, wsR, carB, st);
    launches += 2;
  } else {
    k_encB_rows<<<dim3((unsigned)cdiv(nchB, kThreads / 32), gy(P.nvc)), kThreads, 0, st>>>(
        B, d.ldb, d.k, d.n, d.vb_cols, P.ec, bcs, P.Cc, partB, nchB);
    ++launches;
  }
  k_col_sq<<<dim3((unsigned)cdiv(d.n, kThreads), gy(nchC)), kThreads, 0, st>>>(
      B, d.ldb, d.k, d.n, partC);
  k_sum_sqrt<<<(unsigned)cdiv(d.n, 128), 128, 0, st>>>(partC, d.n, nchC, 1, d.n, nBcol);
  k_finalize_blk<<<(unsigned)cdiv(P.nvr, 128), 128, 0, st>>>(nArow, d.m, d.vb_rows, P.er, partA,
                                                             nchA, nAblk);
  k_finalize_blk<<<(unsigned)cdiv(P.nvc, 128), 128, 0, st>>>(nBcol, d.n, d.vb_cols, P.ec, partB,
                                                             nchB, nBblk);
  count_launches(launches + 5);
  return cudaGetLastError();
}

}  // namespace abft
