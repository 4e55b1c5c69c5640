// Tensor-core ABFT product for bfloat16 operands (Eq. (1)) on sm_103a:
// [A; acs] [B, bcs] with fp32 accumulation in TMEM.
//
// Persistent, warp-specialised kernel, one CTA per SM:
//   warp 0      TMA producer: A tile (128 x 64, K-major) and B tile (64 x 256,
//               N-major, four 64-column boxes) per stage, 128-byte swizzle,
//               into a 4-stage shared-memory ring guarded by mbarriers.
//   warp 1      MMA issuer: one thread issues tcgen05.mma (M=128, N=256,
//               K=16) into one of two TMEM accumulators (2 x 256 columns) and
//               frees ring stages and accumulators with tcgen05.commit.
//   warps 2-5   epilogue: tcgen05.ld of the accumulator (each warp its
//               32-lane quarter), fp32 stores to C or to the checksum
//               outputs, then release of the accumulator so the next tile's
//               MMAs overlap this tile's epilogue.
// Tiles: data tiles (grouped raster for L2 reuse), then checksum-row tiles
// (acs x B -> E16) and checksum-column tiles (A x bcs -> F16); the corner is
// not computed.  Every barrier wait is bounded; a timeout sets a device flag
// the host reports as ABFT_ERR_TIMEOUT, and the kernel still drains its
// copies and MMAs and frees TMEM before returning.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <stdlib.h>

#include <mutex>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace abft {
namespace {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr int kThreads = 192;
constexpr uint32_t A_BYTES = BM * BK * 2;          // 16 KiB
constexpr uint32_t B_BOX_BYTES = 64 * BK * 2;      // one 64-column box: 8 KiB
constexpr uint32_t B_BYTES = BN * BK * 2;          // 32 KiB
constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
constexpr uint32_t TMEM_COLS = 2 * BN;             // two accumulators
constexpr int GROUP_M = 16;                        // tile rows per raster group
constexpr uint32_t OBS_BYTES = 4 * BN * 2 * 4;     // per-warp column partials (e, w)
constexpr size_t SMEM_BYTES = 1024 + STAGES * STAGE_BYTES + OBS_BYTES + 256;

// Tensor maps of the operands: [0] = single / hi plane, [1] = lo plane.  The
// K loop runs over nseg segments of the k dimension; segment s reads A plane
// (s == 2) and B plane (s == 1), so nseg = 3 accumulates
// A_hi B_hi + A_hi B_lo + A_lo B_hi (split bf16x3) and nseg = 1 is plain bf16.
struct TcMaps {
  CUtensorMap a[2], acs[2], b[2], bcs[2];
};

struct TcArgs {
  int64_t m, n, k, R16, C16;
  int nseg;
  int ntm, ntn, ntr, ntc;  // data tile rows/cols, checksum tile rows/cols (0 in plain mode)
  int64_t t_data, t_total;
  float* C;
  int64_t ldc;
  float* E16;  // R16 x n
  float* F16;  // m x C16
  int* status;
  // fused observed checksums of data tiles (nullptr: off)
  float* obs_col;  // [tile row][2][n]
  float* obs_row;  // [row][ngrp][2]
  int vb_r, vb_c, er, ec;
  int64_t g, ngrp;
  const int32_t* inj_hdr;    // armed epilogue injections (nullptr: none)
  const InjectEntry* inj;
  uint64_t wait_ns;          // bounded-wait limit
  int stall_test;            // timeout test: the producer skips the first tile
};

struct Tile {
  int kind;  // 0 data -> C, 1 checksum rows -> E16, 2 checksum columns -> F16
  int64_t row0, col0;
};

// Tile order: groups of GROUP_M data tile rows; the checksum tile rows are
// dealt round-robin to the groups (row r joins group r % groups).  Inside a
// group the tiles run column by column -- data columns over the group's data
// and checksum rows, then the checksum columns over its data rows -- so every
// checksum tile reuses the A or B panels its group already keeps in L2.
__device__ __forceinline__ Tile decode_local(int64_t t, int64_t ntm, int64_t ntn, int64_t ntr,
                                             int64_t ntc) {
  const int64_t ngr = (ntm + GROUP_M - 1) / GROUP_M;
  int64_t off = 0;
  for (int64_t G = 0; G < ngr; ++G) {
    const int64_t gd = min((int64_t)GROUP_M, ntm - G * GROUP_M);
    const int64_t nr = G < ntr ? (ntr - G + ngr - 1) / ngr : 0;
    const int64_t part1 = (gd + nr) * ntn, part2 = gd * ntc;
    if (t < off + part1 + part2) {
      int64_t u = t - off;
      Tile T;
      if (u < part1) {
        const int64_t col = u / (gd + nr), ri = u % (gd + nr);
        T.col0 = col * BN;
        if (ri < gd) {
          T.kind = 0;
          T.row0 = (G * GROUP_M + ri) * BM;
        } else {
          T.kind = 1;
          T.row0 = (G + (ri - gd) * ngr) * BM;
        }
      } else {
        u -= part1;
        T.kind = 2;
        T.col0 = (u / gd) * BN;
        T.row0 = (G * GROUP_M + u % gd) * BM;
      }
      return T;
    }
    off += part1 + part2;
  }
  Tile T;  // not reached for t inside the problem
  T.kind = 0;
  T.row0 = T.col0 = 0;
  return T;
}

__device__ __forceinline__ Tile decode(int64_t t, const TcArgs& g) {
  return decode_local(t, g.ntm, g.ntn, g.ntr, g.ntc);
}

// Everything the three roles need to know about one tile.
struct TileView {
  int kind;                   // 0 data -> C, 1 checksum rows -> E16, 2 checksum columns -> F16
  int prob;                   // problem index (grouped products; 0 otherwise)
  int64_t row0, col0;         // tile origin in its output
  float* dst;                 // output and its leading dimension / limits
  int64_t ld, rlim, clim;
  const CUtensorMap* ma0;     // A-side maps (plane 0 / 1)
  const CUtensorMap* ma1;
  const CUtensorMap* mb0;     // B-side maps
  const CUtensorMap* mb1;
  int64_t nkb;                // k-blocks per segment
  int nseg;
  // fused observed checksums of data tiles (obs_col == nullptr: off)
  float* obs_col;
  float* obs_row;
  int64_t n, m, g, ngrp;
  int vb_r, vb_c, er, ec;
};

// One problem (abft_gemm).
struct SingleSched {
  const TcMaps* M;
  const TcArgs* a;
  __device__ __forceinline__ int64_t total() const { return a->t_total; }
  __device__ __forceinline__ void prefetch() const {
    for (int pl = 0; pl < 2; ++pl) {
      tc::prefetch_tmap(&M->a[pl]);
      tc::prefetch_tmap(&M->acs[pl]);
      tc::prefetch_tmap(&M->b[pl]);
      tc::prefetch_tmap(&M->bcs[pl]);
    }
  }
  __device__ __forceinline__ TileView view(int64_t t) const {
    const TcArgs& g = *a;
    const Tile T = decode(t, g);
    TileView V;
    V.kind = T.kind;
    V.prob = 0;
    V.row0 = T.row0;
    V.col0 = T.col0;
    if (T.kind == 0) { V.dst = g.C; V.ld = g.ldc; V.rlim = g.m; V.clim = g.n; }
    else if (T.kind == 1) { V.dst = g.E16; V.ld = g.n; V.rlim = g.R16; V.clim = g.n; }
    else { V.dst = g.F16; V.ld = g.C16; V.rlim = g.m; V.clim = g.C16; }
    V.ma0 = T.kind == 1 ? &M->acs[0] : &M->a[0];
    V.ma1 = T.kind == 1 ? &M->acs[1] : &M->a[1];
    V.mb0 = T.kind == 2 ? &M->bcs[0] : &M->b[0];
    V.mb1 = T.kind == 2 ? &M->bcs[1] : &M->b[1];
    V.nkb = (g.k + BK - 1) / BK;
    V.nseg = g.nseg;
    V.obs_col = T.kind == 0 ? g.obs_col : nullptr;
    V.obs_row = g.obs_row;
    V.n = g.n;
    V.m = g.m;
    V.g = g.g;
    V.ngrp = g.ngrp;
    V.vb_r = g.vb_r;
    V.vb_c = g.vb_c;
    V.er = g.er;
    V.ec = g.ec;
    return V;
  }
};

__device__ __forceinline__ void store_row32(float* dst, int64_t ld, int64_t row, int64_t col,
                                            int64_t rlim, int64_t clim, const float (&v)[32]) {
  if (row >= rlim) return;
  float* p = dst + row * ld + col;
  if (col + 32 <= clim && ((reinterpret_cast<uintptr_t>(p) & 15) == 0)) {
#pragma unroll
    for (int q = 0; q < 8; ++q)
      reinterpret_cast<float4*>(p)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  } else {
#pragma unroll
    for (int q = 0; q < 32; ++q)
      if (col + q < clim) p[q] = v[q];
  }
}

// Column sums across the 32 lanes of a warp: on return lane l holds, in
// v[0], the sum over all lanes of their element l (31 shuffles).
__device__ __forceinline__ void transpose_reduce(float (&v)[32], int lane) {
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const bool upper = (lane & s) != 0;
#pragma unroll
    for (int i = 0; i < s; ++i) {
      const float send = upper ? v[i] : v[i + s];
      const float keep = upper ? v[i + s] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
}

__device__ __forceinline__ void epi_barrier() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// The kernel body, shared by the single-problem and the grouped product.
template <class Sched>
__device__ __forceinline__ void tc_body(const Sched& S, int* status, uint64_t wait_ns,
                                        int stall_test, const int32_t* inj_hdr,
                                        const InjectEntry* inj) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES + OBS_BYTES);
  // bars[0..S): full, [S..2S): empty, [2S..2S+2): tmem full, [2S+2..2S+4): tmem empty,
  // [2S+4]: drain
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 5);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto full = [&](int s) { return tc::smem_addr(&bars[s]); };
  auto empty = [&](int s) { return tc::smem_addr(&bars[STAGES + s]); };
  auto tfull = [&](int a) { return tc::smem_addr(&bars[2 * STAGES + a]); };
  auto tempty = [&](int a) { return tc::smem_addr(&bars[2 * STAGES + 2 + a]); };
  const uint32_t drain = tc::smem_addr(&bars[2 * STAGES + 4]);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(full(s), 1);
      tc::mbar_init(empty(s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      tc::mbar_init(tfull(a), 1);
      tc::mbar_init(tempty(a), 4);
    }
    tc::mbar_init(drain, 1);
    *abort = 0;
    tc::wait_limit_ns() = wait_ns;
    tc::fence_barrier_init();
    S.prefetch();
  }
  if (warp == 1) {
    tc::tmem_alloc(tc::smem_addr(tmem_slot), TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const int64_t total = S.total();

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer
      int s = 0;
      uint32_t ph = 0;
      int64_t issued = 0;  // stages filled and not known to be consumed
      for (int64_t t = blockIdx.x; t < total && !*abort; t += gridDim.x) {
        const TileView T = S.view(t);
        if (stall_test && t == 0) continue;  // nothing will fill these stages
        const int64_t nkb = T.nkb, nkt = T.nkb * T.nseg;
        for (int64_t kt = 0; kt < nkt; ++kt) {
          const int seg = (int)(kt / nkb);
          const int64_t kb = kt - (int64_t)seg * nkb;
          const CUtensorMap* ma = seg == 2 ? T.ma1 : T.ma0;
          const CUtensorMap* mb = seg == 1 ? T.mb1 : T.mb0;
          if (!tc::wait(empty(s), ph ^ 1, abort)) break;
          const uint32_t sa = tc::smem_addr(smem + s * STAGE_BYTES);
          tc::mbar_arrive_expect_tx(full(s), STAGE_BYTES);
          tc::tma_load_2d(sa, ma, full(s), (int32_t)(kb * BK), (int32_t)T.row0);
#pragma unroll
          for (int c = 0; c < BN / 64; ++c)
            tc::tma_load_2d(sa + A_BYTES + c * B_BOX_BYTES, mb, full(s), (int32_t)(T.col0 + 64 * c),
                            (int32_t)(kb * BK));
          ++issued;
          if (++s == STAGES) { s = 0; ph ^= 1; }
        }
      }
      // Do not leave copies in flight: wait for the last fills (bounded).
      for (int q = 0; q < STAGES && issued > 0; ++q, --issued) {
        if (--s < 0) { s = STAGES - 1; ph ^= 1; }
        const uint64_t t0 = tc::globaltimer();
        while (!tc::mbar_try_wait(full(s), ph) && tc::globaltimer() - t0 < tc::wait_limit_ns()) {
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      constexpr uint32_t idesc = tc::idesc_bf16(BM, BN, 1);
      int s = 0, acc = 0;
      uint32_t ph = 0, aph = 0;
      for (int64_t t = blockIdx.x; t < total && !*abort; t += gridDim.x) {
        const TileView T = S.view(t);
        const int64_t nkt = T.nkb * T.nseg;
        if (!tc::wait(tempty(acc), aph ^ 1, abort)) break;
        tc::fence_after_sync();
        const uint32_t d = tmem + acc * BN;
        bool ok = true;
        for (int64_t kb = 0; kb < nkt; ++kb) {
          if (!tc::wait(full(s), ph, abort)) { ok = false; break; }
          tc::fence_after_sync();
          const uint32_t sa = tc::smem_addr(smem + s * STAGE_BYTES);
          const uint32_t sb = sa + A_BYTES;
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            // A: K-major, 128-byte rows, 8-row groups 1024 B apart; a K step
            // of 16 elements moves 32 B inside the swizzled row.
            const uint64_t ad = tc::sdesc_sw128(sa + kk * 32, 16, 1024);
            // B: N-major, 64-column boxes 8 KiB apart, 8-row (K) groups
            // 1024 B apart; a K step of 16 rows moves 2 KiB.
            const uint64_t bd = tc::sdesc_sw128(sb + kk * 2048, B_BOX_BYTES, 1024);
            tc::mma_f16(d, ad, bd, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
          }
          tc::commit(empty(s));
          if (++s == STAGES) { s = 0; ph ^= 1; }
        }
        if (!ok) break;
        tc::commit(tfull(acc));
        if (++acc == 2) { acc = 0; aph ^= 1; }
      }
      // Every MMA issued so far must complete before TMEM is freed.
      tc::commit(drain);
      const uint64_t t0 = tc::globaltimer();
      while (!tc::mbar_try_wait(drain, 0) && tc::globaltimer() - t0 < tc::wait_limit_ns()) {
      }
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: warps 2..5, TMEM lane quarter = warp % 4
    const int q = warp & 3;
    float* obs = reinterpret_cast<float*>(smem + STAGES * STAGE_BYTES);  // [4][BN][2]
    const int ninj = (inj_hdr && inj_hdr[0] == kInjectMagic)
                         ? max(0, min(inj_hdr[1], kMaxInject)) : 0;
    int acc = 0;
    uint32_t aph = 0;
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
      const TileView T = S.view(t);
      if (!tc::wait(tfull(acc), aph, abort)) break;
      tc::fence_after_sync();
      float* const dst = T.dst;
      const int64_t ld = T.ld, rlim = T.rlim, clim = T.clim;
      const int64_t row = T.row0 + q * 32 + lane;
      const bool fused = T.obs_col != nullptr;
      const float scr = scalbnf(1.0f, -T.er), scc = scalbnf(1.0f, -T.ec);
      const float wrow = fused ? (float)((int)(row % T.vb_r) + 1) * scr : 0.f;
      float racc_e = 0.f, racc_w = 0.f;
      const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + acc * BN;
#pragma unroll 1
      for (int c = 0; c < BN; c += 32) {
        float v[32];
        tc::tmem_ld32(base + c, v);
        if (T.col0 + c >= clim) continue;
        const int64_t col = T.col0 + c;
        if (T.kind == 0)
          for (int f = 0; f < ninj; ++f) {
            const InjectEntry ie = inj[f];
            if (ie.pad == T.prob && ie.row == row && ie.col >= col && ie.col < col + 32) {
              const int x = ie.col - (int)col;
#pragma unroll
              for (int u = 0; u < 32; ++u)
                if (u == x) v[u] = __uint_as_float(__float_as_uint(v[u]) ^ (1u << (ie.bit & 31)));
            }
          }
        store_row32(dst, ld, row, col, rlim, clim, v);
        if (fused) {
          // row partials over the column group (weights restart per verify block;
          // a 32-column chunk never straddles one)
          const int cm = (int)(col % T.vb_c) + 1;
#pragma unroll
          for (int u = 0; u < 32; ++u) {
            racc_e += v[u];
            racc_w = fmaf((float)(cm + u) * scc, v[u], racc_w);
          }
          if (((c + 32) % (int)T.g) == 0 || c + 32 == BN || col + 32 >= clim) {
            if (row < T.m) {
              float* o = T.obs_row + (row * T.ngrp + (int)(col / T.g)) * 2;
              o[0] = racc_e;
              o[1] = racc_w;
            }
            racc_e = racc_w = 0.f;
          }
          // column partials of this warp's 32 rows
          float vw[32];
#pragma unroll
          for (int u = 0; u < 32; ++u) vw[u] = wrow * v[u];
          transpose_reduce(v, lane);
          transpose_reduce(vw, lane);
          obs[(q * BN + c + lane) * 2 + 0] = v[0];
          obs[(q * BN + c + lane) * 2 + 1] = vw[0];
        }
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(tempty(acc));
      if (++acc == 2) { acc = 0; aph ^= 1; }
      if (fused) {
        epi_barrier();
        const int et = q * 32 + lane;  // 0..127
        const int64_t tr = T.row0 / BM;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int cc = et + h * 128;
          const int64_t col = T.col0 + cc;
          if (col < T.n) {
            float se = 0.f, sw = 0.f;
#pragma unroll
            for (int w4 = 0; w4 < 4; ++w4) {
              se += obs[(w4 * BN + cc) * 2 + 0];
              sw += obs[(w4 * BN + cc) * 2 + 1];
            }
            T.obs_col[(tr * 2 + 0) * T.n + col] = se;
            T.obs_col[(tr * 2 + 1) * T.n + col] = sw;
          }
        }
        epi_barrier();
      }
    }
  }

  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x == 0 && *abort) atomicExch(status, 1);
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, TMEM_COLS);
  }
}

__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_bf16(const __grid_constant__ TcMaps M, const TcArgs g) {
  const SingleSched S{&M, &g};
  tc_body(S, g.status, g.wait_ns, g.stall_test, g.inj_hdr, g.inj);
}

// Many problems (grouped product): the flattened tile list is the problems'
// tile lists one after the other; per-problem tables and tensor maps live in
// global memory.  Verify blocks equal the tile (128 x 256).
struct GroupSched {
  const GProb* probs;
  const GMaps* maps;
  int count;
  int64_t t_total;
  bool checksums;
  __device__ __forceinline__ int64_t total() const { return t_total; }
  __device__ __forceinline__ void prefetch() const {}
  __device__ __forceinline__ TileView view(int64_t t) const {
    int lo = 0, hi = count - 1;  // last problem with tile_off <= t
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (probs[mid].tile_off <= t) lo = mid; else hi = mid - 1;
    }
    const GProb& P = probs[lo];
    const GMaps& Mp = maps[lo];
    const Tile T = checksums ? decode_local(t - P.tile_off, P.ntm, P.ntn, P.ntr, P.ntc)
                             : decode_local(t - P.tile_off, P.ntm, P.ntn, 0, 0);
    TileView V;
    V.kind = T.kind;
    V.prob = lo;
    V.row0 = T.row0;
    V.col0 = T.col0;
    if (T.kind == 0) { V.dst = P.C; V.ld = P.ldc; V.rlim = P.m; V.clim = P.n; }
    else if (T.kind == 1) { V.dst = P.E16; V.ld = P.n; V.rlim = P.R16; V.clim = P.n; }
    else { V.dst = P.F16; V.ld = P.C16; V.rlim = P.m; V.clim = P.C16; }
    V.ma0 = V.ma1 = T.kind == 1 ? &Mp.acs : &Mp.a;
    V.mb0 = V.mb1 = T.kind == 2 ? &Mp.bcs : &Mp.b;
    V.nkb = (P.k + BK - 1) / BK;
    V.nseg = 1;
    V.obs_col = (T.kind == 0 && checksums) ? P.obs_col : nullptr;
    V.obs_row = P.obs_row;
    V.n = P.n;
    V.m = P.m;
    V.g = kGrpVbC;
    V.ngrp = P.nvc;
    V.vb_r = kGrpVbR;
    V.vb_c = kGrpVbC;
    V.er = 7;
    V.ec = 8;
    return V;
  }
};

__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_grouped(const GProb* probs, const GMaps* maps, int count, int64_t t_total,
                   int checksums, int* status, uint64_t wait_ns, const int32_t* inj_hdr,
                   const InjectEntry* inj) {
  const GroupSched S{probs, maps, count, t_total, checksums != 0};
  tc_body(S, status, wait_ns, 0, inj_hdr, inj);
}

// ---- host side
PFN_cuTensorMapEncodeTiled_v12000 g_encode_tiled = nullptr;
std::once_flag g_encode_once;
int g_num_sms[64] = {};

cudaError_t get_encoder() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode_tiled = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  return g_encode_tiled ? cudaSuccess : cudaErrorNotSupported;
}

// 2-D bf16 tensor map over a row-major rows x cols matrix with leading
// dimension ld (elements), box of box_cols x box_rows, 128-byte swizzle.
bool make_map(CUtensorMap* map, const void* ptr, int64_t rows, int64_t cols, int64_t ld,
              uint32_t box_cols, uint32_t box_rows) {
  if (rows == 0 || cols == 0) {  // never read: a dummy valid map
    rows = 1;
    cols = 8;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  const cuuint32_t box[2] = {box_cols, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return g_encode_tiled(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int num_sms() {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 148;
  if (!g_num_sms[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    g_num_sms[dev] = v > 0 ? v : 148;
  }
  return g_num_sms[dev];
}

}  // namespace

// Device flag set by a tensor-core product whose bounded waits gave up.
__device__ int g_tc_timeout = 0;

cudaError_t tc_timeout_flag(int** dev_ptr) {
  return cudaGetSymbolAddress(reinterpret_cast<void**>(dev_ptr), g_tc_timeout);
}

// Reads and clears the timeout flag, stream-ordered (synchronises `st`).
cudaError_t consume_tc_timeout(cudaStream_t st, bool* timed_out) {
  int* flag = nullptr;
  cudaError_t e = tc_timeout_flag(&flag);
  int v = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&v, flag, sizeof v, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && v) e = cudaMemsetAsync(flag, 0, sizeof(int), st);
  *timed_out = v != 0;
  return e;
}

cudaError_t launch_gemm_bf16(const Plan& P, const TcOperands& op, float* C, void* ws,
                             bool checksums, cudaStream_t st) {
  cudaError_t e = get_encoder();
  if (e != cudaSuccess) return e;
  const abft_desc& d = P.d;
  const char* w = static_cast<const char*>(ws);
  const int64_t R16 = checksums ? P.L.acs_rows : 0, C16 = checksums ? P.L.bcs_cols : 0;
  TcMaps M;
  for (int pl = 0; pl < 2; ++pl) {
    const void* acs = checksums ? w + P.L.acs + pl * P.L.acs_plane : op.a[0];
    const void* bcs = checksums ? w + P.L.bcs + pl * P.L.bcs_plane : op.b[0];
    if (!make_map(&M.a[pl], op.a[pl], d.m, d.k, op.lda, 64, BM) ||
        !make_map(&M.acs[pl], acs, R16, d.k, checksums ? P.L.acs_ld : op.lda, 64, BM) ||
        !make_map(&M.b[pl], op.b[pl], d.k, d.n, op.ldb, 64, BK) ||
        !make_map(&M.bcs[pl], bcs, d.k, C16, checksums ? P.L.bcs_ld : op.ldb, 64, BK))
      return cudaErrorInvalidValue;
  }
  TcArgs g{};
  g.m = d.m; g.n = d.n; g.k = d.k; g.R16 = R16; g.C16 = C16;
  g.nseg = op.nseg;
  g.ntm = (int)cdiv(d.m, BM);
  g.ntn = (int)cdiv(d.n, BN);
  g.ntr = checksums ? (int)cdiv(R16, BM) : 0;
  g.ntc = checksums ? (int)cdiv(C16, BN) : 0;
  g.t_data = (int64_t)g.ntm * g.ntn;
  g.t_total = g.t_data + (int64_t)g.ntr * g.ntn + (int64_t)g.ntm * g.ntc;
  g.C = C;
  g.ldc = d.ldc;
  g.E16 = checksums ? reinterpret_cast<float*>(const_cast<char*>(w) + P.L.E16) : nullptr;
  g.F16 = checksums ? reinterpret_cast<float*>(const_cast<char*>(w) + P.L.F16) : nullptr;
  g.vb_r = d.vb_rows;
  g.vb_c = d.vb_cols;
  g.er = P.er;
  g.ec = P.ec;
  g.g = P.g > 0 ? P.g : 256;
  g.ngrp = P.ngrp;
  if (checksums && P.fused) {
    g.obs_col = reinterpret_cast<float*>(const_cast<char*>(w) + P.L.obs_col);
    g.obs_row = reinterpret_cast<float*>(const_cast<char*>(w) + P.L.obs_row);
  }
  if (checksums) {
    g.inj_hdr = reinterpret_cast<const int32_t*>(w + P.L.inject);
    g.inj = reinterpret_cast<const InjectEntry*>(w + P.L.inject + 16);
  }
  e = tc_timeout_flag(&g.status);
  if (e != cudaSuccess) return e;
  // Test hook for the bounded waits: ABFT_TEST_STALL_PRODUCER=1 makes the
  // producer skip the first tile, so its MMA wait runs out (after 0.2 s) and
  // the call reports ABFT_ERR_TIMEOUT.  Off unless the variable is set.
  const char* stall = getenv("ABFT_TEST_STALL_PRODUCER");
  g.stall_test = stall && stall[0] == '1';
  g.wait_ns = g.stall_test ? 200000000ull : tc::kWaitLimitNs;
  e = cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)SMEM_BYTES);
  if (e != cudaSuccess) return e;
  const int grid = (int)std::min<int64_t>(g.t_total, num_sms());
  if (grid == 0) return cudaSuccess;
  k_gemm_bf16<<<grid, kThreads, SMEM_BYTES, st>>>(M, g);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t make_bf16_map(CUtensorMap* map, const void* ptr, int64_t rows, int64_t cols,
                          int64_t ld, uint32_t box_cols, uint32_t box_rows) {
  cudaError_t e = get_encoder();
  if (e != cudaSuccess) return e;
  return make_map(map, ptr, rows, cols, ld, box_cols, box_rows) ? cudaSuccess
                                                                : cudaErrorInvalidValue;
}

cudaError_t launch_gemm_grouped(const GProb* probs, const GMaps* maps, int count,
                                int64_t t_total, bool checksums, const int32_t* inj_hdr,
                                const InjectEntry* inj, cudaStream_t st) {
  int* status = nullptr;
  cudaError_t e = tc_timeout_flag(&status);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_gemm_grouped, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)SMEM_BYTES);
  if (e != cudaSuccess) return e;
  const int grid = (int)std::min<int64_t>(t_total, num_sms());
  if (grid == 0) return cudaSuccess;
  k_gemm_grouped<<<grid, kThreads, SMEM_BYTES, st>>>(probs, maps, count, t_total,
                                                     checksums ? 1 : 0, status,
                                                     tc::kWaitLimitNs, inj_hdr, inj);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace abft
