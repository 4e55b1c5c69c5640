// Binary64 ABFT product (Eq. (1)): [A; acs] [B, bcs] on the FP64 FMA pipe.
//
// On GB300 the FP64 FMA pipe issues 2 DFMA per clock per SM (measured
// 1.20 TFLOP/s over 152 SMs); mma.sync f64 runs slower (1.05 TFLOP/s) and
// tcgen05 has no f64 kind, so the kernel is a shared-memory tiled DFMA GEMM
// whose only job is to keep that pipe busy.  A 64x64 tile per 256-thread CTA,
// 4x4 outputs per thread, BK = 16 with a register-prefetched double buffer.
// Memory traffic is ~(1/64 + 1/64) words per FMA, far below HBM and L2
// bandwidth at this FMA rate.
//
// Tiles are scheduled as one 1-D grid in a grouped order (see decode_f64):
// data tiles, whole tiles of checksum rows (acs, writing E) and checksum
// columns (bcs, writing F); the corner (acs x bcs) is not computed.  Each output element is one FMA chain
// over k in increasing order.
#include "internal.cuh"

namespace abft {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, kThreads = 256;

constexpr int GROUP_M = 16;  // tile rows per raster group

struct GemmArgs {
  const double* A;
  const double* B;
  const double* acs;
  const double* bcs;
  double* C;
  double* E;
  double* F;
  int64_t lda, ldb, ldc, m, n, k, R, Cc;
  int tm, tn;  // data tiles along rows / columns
  int tr, tc;  // checksum tiles along rows / columns (0 for the plain product)
};

// Linear tile index -> (tile row, tile column), tile rows >= tm being checksum
// rows and tile columns >= tn checksum columns.  Groups of GROUP_M data tile
// rows run column by column; checksum tile rows are dealt round-robin to the
// groups and checksum tile columns follow each group's data columns, so
// consecutive CTAs share the A and B panels in L2.
__device__ __forceinline__ void decode_f64(int64_t t, const GemmArgs& g, int& ty, int& tx) {
  const int64_t ngr = (g.tm + GROUP_M - 1) / GROUP_M;
  int64_t off = 0;
  for (int64_t G = 0; G < ngr; ++G) {
    const int64_t gd = min((int64_t)GROUP_M, (int64_t)g.tm - G * GROUP_M);
    const int64_t nr = G < g.tr ? (g.tr - G + ngr - 1) / ngr : 0;
    const int64_t part1 = (gd + nr) * g.tn, part2 = gd * g.tc;
    if (t < off + part1 + part2) {
      int64_t u = t - off;
      if (u < part1) {
        const int64_t ri = u % (gd + nr);
        tx = (int)(u / (gd + nr));
        ty = ri < gd ? (int)(G * GROUP_M + ri) : (int)(g.tm + G + (ri - gd) * ngr);
      } else {
        u -= part1;
        tx = (int)(g.tn + u / gd);
        ty = (int)(G * GROUP_M + u % gd);
      }
      return;
    }
    off += part1 + part2;
  }
  ty = tx = 0;
}

__global__ void __launch_bounds__(kThreads, 2) k_gemm_f64(const GemmArgs g) {
  int ty_tile, tx_tile;
  decode_f64(blockIdx.x, g, ty_tile, tx_tile);
  const bool cs_row = ty_tile >= g.tm, cs_col = tx_tile >= g.tn;

  // Source and destination of this tile.
  const double* Asrc;
  int64_t ldA, rlim, row0;
  if (!cs_row) {
    Asrc = g.A; ldA = g.lda; rlim = g.m; row0 = (int64_t)ty_tile * BM;
  } else {
    Asrc = g.acs; ldA = g.k; rlim = g.R; row0 = (int64_t)(ty_tile - g.tm) * BM;
  }
  const double* Bsrc;
  int64_t ldB, clim, col0;
  if (!cs_col) {
    Bsrc = g.B; ldB = g.ldb; clim = g.n; col0 = (int64_t)tx_tile * BN;
  } else {
    Bsrc = g.bcs; ldB = g.Cc; clim = g.Cc; col0 = (int64_t)(tx_tile - g.tn) * BN;
  }
  double* Dst;
  int64_t ldD;
  if (!cs_row && !cs_col) { Dst = g.C; ldD = g.ldc; }
  else if (cs_row) { Dst = g.E; ldD = g.n; }
  else { Dst = g.F; ldD = g.Cc; }

  __shared__ double As[2][BK][BM + 2];
  __shared__ double Bs[2][BK][BN];

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  double ra[4], rb[4];
  auto load = [&](int64_t k0) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = e * kThreads + tid;
      const int r = idx >> 4, c = idx & 15;
      const int64_t row = row0 + r, kk = k0 + c;
      ra[e] = (row < rlim && kk < g.k) ? Asrc[row * ldA + kk] : 0.0;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = e * kThreads + tid;
      const int r = idx >> 6, c = idx & 63;
      const int64_t kk = k0 + r, col = col0 + c;
      rb[e] = (kk < g.k && col < clim) ? Bsrc[kk * ldB + col] : 0.0;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = e * kThreads + tid;
      As[buf][idx & 15][idx >> 4] = ra[e];
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = e * kThreads + tid;
      Bs[buf][idx >> 6][idx & 63] = rb[e];
    }
  };

  const int64_t nk = cdiv(g.k, BK);
  load(0);
  store(0);
  __syncthreads();
  int buf = 0;
  for (int64_t kt = 0; kt < nk; ++kt) {
    if (kt + 1 < nk) load((kt + 1) * BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    if (kt + 1 < nk) store(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }

#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t row = row0 + ty + 16 * i;
    if (row >= rlim) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t col = col0 + tx + 16 * j;
      if (col < clim) Dst[row * ldD + col] = acc[i][j];
    }
  }
}

}  // namespace

cudaError_t launch_gemm_f64(const Plan& P, const double* A, const double* B, double* C, void* ws,
                            bool checksums, cudaStream_t st) {
  const abft_desc& d = P.d;
  GemmArgs g{};
  g.A = A; g.B = B; g.C = C;
  g.lda = d.lda; g.ldb = d.ldb; g.ldc = d.ldc;
  g.m = d.m; g.n = d.n; g.k = d.k;
  g.tm = (int)cdiv(d.m, BM);
  g.tn = (int)cdiv(d.n, BN);
  if (checksums) {
    char* w = static_cast<char*>(ws);
    g.acs = reinterpret_cast<const double*>(w + P.L.acs);
    g.bcs = reinterpret_cast<const double*>(w + P.L.bcs);
    g.E = reinterpret_cast<double*>(w + P.L.E);
    g.F = reinterpret_cast<double*>(w + P.L.F);
    g.R = P.R;
    g.Cc = P.Cc;
    g.tr = (int)cdiv(P.R, BM);
    g.tc = (int)cdiv(P.Cc, BN);
  }
  if (d.m == 0 || d.n == 0) return cudaSuccess;
  const int64_t tiles = (int64_t)g.tm * g.tn + (int64_t)g.tr * g.tn + (int64_t)g.tm * g.tc;
  k_gemm_f64<<<(unsigned)tiles, kThreads, 0, st>>>(g);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace abft
