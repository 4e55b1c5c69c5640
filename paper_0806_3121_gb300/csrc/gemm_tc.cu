// Tensor-core ABFT product for bfloat16 operands (Eq. (1)) on sm_103a:
// [A; acs] [B, bcs] with fp32 accumulation in TMEM.
//
// Persistent, warp-specialised kernel, one CTA per SM:
//   warp 0      TMA producer of A: one 128-row box (or two 64-row halves) per
//               stage, K-major, 128-byte swizzle, into a 4-stage shared-memory
//               ring guarded by mbarriers (256-row tiles: two 128-row boxes,
//               3 stages; see Geo).
//   warp 10     TMA producer of B: one 3-D copy of up to four 64-column boxes
//               (N-major) per stage, the ragged / checksum boxes one by one; the
//               two producers arrive on a stage's full barrier with their own
//               bytes (one issuing thread could not keep up with the MMAs).
//   warp 1      MMA issuer: one thread issues tcgen05.mma (M=128, N=64 x boxes,
//               K=16) into one of two TMEM accumulators (2 x 256 columns; a
//               256-row tile uses both, one per 128-row half) and frees ring
//               stages and accumulators with tcgen05.commit.
//   warps 2-9   epilogue: tcgen05.ld of the accumulator (a warp reads its
//               32-lane quarter of TMEM and one 128-column half of the tile;
//               on 256-row tiles one 128-row accumulator, all 256 columns),
//               each 32 x 32 chunk staged in shared memory and written to C or
//               the checksum outputs by a TMA store, the fused observed sums,
//               then release of the accumulator so the next tile's MMAs
//               overlap this tile's epilogue (on 128-row tiles).
// Single problem: data tiles (grouped raster for L2 reuse), checksum-row tiles
// (acs x B -> E16) and checksum-column tiles (A x bcs -> F16); the corner is
// not computed.  Grouped problems: each problem's checksum halves / boxes
// follow its data halves / boxes and share the last data tiles.  Every barrier wait is bounded; a timeout sets a device flag
// of the workspace that the host reports as ABFT_ERR_TIMEOUT, and the kernel still drains its
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
#ifndef ABFT_EPI_WARPS
#define ABFT_EPI_WARPS 8
#endif
constexpr int kEpiWarps = ABFT_EPI_WARPS;         // 4 or 8 (one or two per TMEM lane quarter)
constexpr int kEpiCols = BN * 4 / kEpiWarps;       // tile columns per epilogue warp
constexpr int kEpiChunks = kEpiCols / 32;          // 32-column TMEM loads per warp
// warps: 0 TMA producer of A, 1 MMA issuer, 2 .. 1 + kEpiWarps epilogue (warp
// w reads TMEM lane quarter w % 4), then the TMA producer of B
constexpr int kWarpProdB = 2 + kEpiWarps;
constexpr int kThreads = 32 * (kWarpProdB + 1);
// Every epilogue warp reads whole 32-column chunks of its TMEM lane quarter:
// a split that is not a multiple of 32 columns would read past the
// accumulator (and past the allocated TMEM for the second one).
static_assert(kEpiWarps == 4 || kEpiWarps == 8, "4 or 8 epilogue warps");
static_assert((BN * 4) % kEpiWarps == 0 && kEpiCols % 32 == 0, "whole 32-column chunks");
constexpr uint32_t A_BYTES = BM * BK * 2;          // 16 KiB
constexpr uint32_t HALF_BYTES = 64 * BK * 2;       // one 64-row half of A: 8 KiB
constexpr uint32_t B_BOX_BYTES = 64 * BK * 2;      // one 64-column box: 8 KiB
constexpr uint32_t B_BYTES = BN * BK * 2;          // 32 KiB
// FP8 data tiles: a k-step is 128 e4m3 codes (the same 128 bytes per row as a
// bf16 k-step, so the stage layout is unchanged); B is read K-major from its
// transposed copy, 64 columns of C (64 rows of B^T, 8 KiB) per box
constexpr int BK8 = 128;
constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
constexpr uint32_t TMEM_COLS = 2 * BN;             // two accumulators
constexpr uint32_t STG_BYTES = 32 * 32 * 4;        // one epilogue warp's staging block
constexpr size_t SMEM_BYTES = 1024 + STAGES * STAGE_BYTES + kEpiWarps * STG_BYTES + 256;
static_assert(SMEM_BYTES <= 232448, "shared memory per CTA");

// Tile geometry.  Regular tiles are 128 x 256 with two accumulators that
// alternate between tiles (the epilogue of one tile overlaps the MMAs of the
// next).  Tall tiles are 256 x 256: two M = 128 MMAs per K step share the B
// stage, one accumulator per 128-row half (both halves of TMEM), so the
// operand bytes per flop fall by a third and the ring holds 3 stages of
// 64 KiB; the epilogue no longer overlaps the next tile's MMAs, which pays
// off for long K loops.  Pair tiles are 256 x 256 on a CTA pair (a cluster of
// two): one M = 256 MMA per K step (cta_group::2) reads 128 rows of A and
// 128 columns of B from each CTA's ring, so each CTA stages 32 KiB per K step
// (the tall tile's bytes per flop) in a 6-stage ring and keeps its 128 rows
// of the tile in TMEM with two alternating accumulators (the regular tile's
// overlapped epilogue).
template <bool kTall, bool kPair = false>
struct Geo {
  static_assert(!(kTall && kPair), "tall or pair tiles");
  static constexpr int kBM = (kTall || kPair) ? 256 : BM;   // rows of the scheduled tile
  static constexpr int kStages = kTall ? 3 : (kPair ? 6 : STAGES);
  static constexpr uint32_t kABytes = (uint32_t)(kTall ? 256 : BM) * BK * 2;  // this CTA's A
  static constexpr uint32_t kBBytes = kPair ? B_BYTES / 2 : B_BYTES;         // this CTA's B
  static constexpr uint32_t kStageBytes = kABytes + kBBytes;
  static constexpr int kSlots = kTall ? 1 : 2;            // accumulator slots that alternate
  static constexpr int kCols = kTall ? BN : kEpiCols;     // tile columns per epilogue warp
  static constexpr size_t kSmem =
      1024 + (size_t)kStages * kStageBytes + kEpiWarps * STG_BYTES + 256;
};
static_assert(Geo<false>::kSmem == SMEM_BYTES, "regular tiles");
static_assert(Geo<true>::kSmem <= 232448, "shared memory per CTA (tall tiles)");
static_assert(Geo<false, true>::kSmem <= 232448, "shared memory per CTA (pair tiles)");
static_assert(Geo<true>::kBM / 128 * BN <= (int)TMEM_COLS, "tall accumulators fit TMEM");

// Tensor maps of the operands, per bf16 plane (the split dtypes have 2 or 3
// planes; unused planes repeat plane 0).  The K loop runs nseg segments;
// segment s reads A plane (seg_a >> 2s) & 3 and B plane (seg_b >> 2s) & 3.
constexpr int kPlanes = 3;
// Native FP8 data tiles read the e4m3 codes, both K-major: A as 64-row halves
// (a[kF8Slot]) and 128-row boxes (a128[kF8Slot]) of 128 codes, B's transposed
// copy B^T (n x k) as 64-row boxes (b[kF8Slot]) and the 256-row box of a full
// tile (b4[kF8Slot]).  They take the plane-1 slots, which an FP8 product does
// not use (its checksum tiles read plane 0), so the kernel parameters stay
// within 4 KiB.
constexpr int kF8Slot = 1;
struct TcMaps {
  CUtensorMap a[kPlanes], acs[kPlanes], b[kPlanes], bcs[kPlanes], a128[kPlanes],
      acs128[kPlanes], b4[kPlanes], bcs4[kPlanes];
  CUtensorMap cst, est, fst;  // fp32 store maps of C, E16, F16 (valid per TcArgs::st_ok)
};

struct TcArgs {
  int64_t m, n, k, R16, C16;
  int nseg;
  uint32_t seg_a, seg_b;
  int ntm, ntn, ntr, ntc;  // data tile rows/cols, checksum tile rows/cols (0 in plain mode)
  int64_t t_data, t_total;
  float* C;
  int64_t ldc;
  float* E16;  // R16 x n
  float* F16;  // m x C16
  int* status;
  // fused observed checksums of data tiles (nullptr: off)
  float* obs_col;  // [32-row block][2][n]
  float* obs_row;  // [row][ngrp][2]
  int st_ok;       // bit 0/1/2: TMA store map of C / E16 / F16 valid
  int vb_r, vb_c, er, ec;
  int64_t g, ngrp;
  const int32_t* inj_hdr;    // armed epilogue injections (nullptr: none)
  const InjectEntry* inj;
  uint64_t wait_ns;          // bounded-wait limit
  int stall_test;            // timeout test: the producer skips the first tile
  int kpg;                   // k-steps per promotion group (0: one group per tile)
  int group_m;               // raster group height (tile rows)
  // native FP8 data tiles: e4m3 products on the 8-bit tensor path, one
  // 128-wide k-step per accumulator, each scaled in the epilogue by the
  // power-of-two block scales sA[row block][k block] * sB[k block][column block]
  int f8;
  const float* sA;           // ceil(m/128) x nsa
  const float* sB;           // ceil(k/128) x nsb
  int64_t nsa, nsb;
  // scale groups of every data tile: bit kb of its f8words words is set when
  // k-step kb starts a new group (the block-scale product of either 128-column
  // half of the tile differs from k-step kb - 1's); a group accumulates in one
  // TMEM accumulator and is scaled once
  const uint32_t* f8grp;
  int64_t f8words;
  int64_t cs_stride;         // FP8 tile order: checksum tile c at position c * cs_stride
};

// The product kernel's parameters (tensor maps and arguments, passed by value
// as __grid_constant__ and copied at every launch) stay within the classic
// 4 KiB parameter space.
static_assert(sizeof(TcMaps) + sizeof(TcArgs) <= 4096, "kernel parameters within 4 KiB");

struct Tile {
  int kind;  // 0 data -> C, 1 checksum rows -> E16, 2 checksum columns -> F16
  int64_t row0, col0;
};

// Tile order: groups of GROUP_M (raster group height) data tile rows; the checksum tile rows are
// dealt round-robin to the groups (row r joins group r % groups).  Inside a
// group the tiles run column by column -- data columns over the group's data
// and checksum rows, then the checksum columns over its data rows -- so every
// checksum tile reuses the A or B panels its group already keeps in L2.
__device__ __forceinline__ Tile decode_local(int64_t t, int64_t ntm, int64_t ntn, int64_t ntr,
                                             int64_t ntc, int64_t GROUP_M, int64_t bm) {
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
          T.row0 = (G * GROUP_M + ri) * bm;
        } else {
          T.kind = 1;
          T.row0 = (G + (ri - gd) * ngr) * bm;
        }
      } else {
        u -= part1;
        T.kind = 2;
        T.col0 = (u / gd) * BN;
        T.row0 = (G * GROUP_M + u % gd) * bm;
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

// Tile order of products with native FP8 data tiles: their checksum tiles run
// on the bf16 planes (twice as long per tile, sharing no operand with the data
// tiles, so their panels come from DRAM), so they are spread through the
// first part of the schedule: checksum tile c (the checksum-row tiles first,
// the two of a tile column back to back, then the checksum-column tiles) sits
// at flat position c * S, the data tiles fill the other positions in the
// grouped raster of the data alone.  S is coprime with the grid, so the
// round-robin assignment gives every CTA at most ceil(checksum tiles / grid)
// of them, at different times (S = 1: all checksum tiles first).
__device__ __forceinline__ Tile decode_cs_spread(int64_t t, int64_t ntm, int64_t ntn, int64_t ntr,
                                                 int64_t ntc, int64_t GROUP_M, int64_t bm,
                                                 int64_t S) {
  const int64_t n1 = ntr * ntn, n2 = ntm * ntc, ncs = n1 + n2;
  if (t % S == 0 && t / S < ncs) {
    const int64_t c = t / S;
    Tile T;
    if (c < n1) {
      T.kind = 1;
      T.row0 = (c % ntr) * bm;
      T.col0 = (c / ntr) * BN;
    } else {
      const int64_t u = c - n1;
      T.kind = 2;
      T.row0 = (u % ntm) * bm;
      T.col0 = (u / ntm) * BN;
    }
    return T;
  }
  const int64_t before = min(ncs, t / S + 1);  // checksum positions at or before t
  return decode_local(t - before, ntm, ntn, 0, 0, GROUP_M, bm);
}

__device__ __forceinline__ int64_t clamp64(int64_t v, int64_t lo, int64_t hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

// Everything the three roles need to know about one tile.  The A operand of a
// tile is two 64-row halves and its B operand nbox 64-column boxes; each half
// (box) comes either from the data operand or from its checksum operand, so a
// tile can hold data rows and checksum rows (columns) side by side:
//   halves [0, hsplit)     data rows      rowD + 64 h           -> C / F16
//   halves [hsplit, hcnt)  checksum rows  rowC + 64 (h-hsplit)  -> E16
//   boxes  [0, bsplit)     data columns   colD + 64 b           -> C / E16
//   boxes  [bsplit, nbox)  checksum cols  colC + 64 (b-bsplit)  -> F16
// checksum row x checksum column products (the corner) are not stored.
struct TileView {
  int prob;                   // problem index (grouped products; 0 otherwise)
  int64_t nkb;                // k-blocks per segment
  int nseg;
  int kpg;                    // k-steps per promotion group (0: the whole K loop)
  uint32_t seg_a, seg_b;      // plane of A / B per K segment (2 bits each)
  const CUtensorMap* maD;     // A-side maps: data / checksum (plane p at + p)
  const CUtensorMap* maC;
  const CUtensorMap* mbD;     // B-side maps
  const CUtensorMap* mbC;
  int32_t rowD, rowC, colD, colC;
  int hsplit, hcnt, bsplit, nbox;
  int nmma;                   // MMA N: 64 nbox, or less when the last box is a checksum
                              // box with fewer used columns (see mma_cols)
  // swapped checksum-row tile (grouped products, kGrpSwapTile): E16 columns
  // colW .. colW + 255 as the M side of two M = 128 MMAs (four B boxes from mbW
  // / mbD, in the B region), the R16 checksum rows as their N side (nsw_h
  // 64-row halves of acs from maC, in the A region), MMA N = nsw_n <= 128; the
  // epilogue stores the accumulators transposed into E16
  int swap, nsw_h, nsw_n;
  // k-steps per ring stage: 1, or 2 for a grouped checksum-column tile
  // (kGrpF2Tile: A of k-step 1 in the first 16 KiB of the B region, the
  // checksum boxes of k-steps 0 / 1 at 16 / 24 KiB of it)
  int k2;
  // one-copy loads: A as nA128 128-row boxes (maW, rows rowW + 128 i) and
  // full B boxes (mbW: 3-D map at box index colW / 64); nullptr: per half / box
  const CUtensorMap* maW;     // (plane p at + p)
  const CUtensorMap* mbW;     // boxes [0, nW) in one copy; the rest per box
  int32_t rowW, colW, nW;
  int nA128;
  float* C;                   // data x data, ld ldc, m x n
  int64_t ldc, m, n;
  float* E16;                 // checksum rows x data columns, ld n, R16 rows
  int64_t R16;
  float* F16;                 // data rows x checksum columns, ld C16
  int64_t C16;
  // TMA store maps of the three outputs (nullptr: plain stores)
  const CUtensorMap* sC;
  const CUtensorMap* sE;
  const CUtensorMap* sF;
  // fused observed checksums of data tiles (obs_col == nullptr: off)
  float* obs_col;             // [32-row block][2][n]
  float* obs_row;             // [row][ngrp][2]
  int64_t g, ngrp;
  int vb_r, vb_c, er, ec;
  // native FP8 data tile: k-steps of 128 e4m3 codes (maD / maW / mbD / mbW are
  // the e4m3 maps), each promoted with the scale sArow[kb] * sB[kb * nsb + J]
  bool f8;
  const float* sArow;
  const float* sB;
  int64_t nsb;
  const uint32_t* gmask;      // this tile's scale-group words (see TcArgs::f8grp)
  // 256-row tiles: the scales and group words of rows row0 + 128 .. (nullptr
  // when those rows are past the data)
  const float* sArow2;
  const uint32_t* gmask2;
};

// End of the scale group that starts at k-step kb: the next k-step whose bit is
// set in the tile's group words, or nkt.
__device__ __forceinline__ int64_t group_end(const uint32_t* mask, int64_t kb, int64_t nkt) {
  int64_t x = kb + 1;
  while (x < nkt) {
    const uint32_t w = __ldg(&mask[x >> 5]) >> (x & 31);
    if (w) {
      const int64_t e = x + __ffs(w) - 1;
      return e < nkt ? e : nkt;
    }
    x = (x | 31) + 1;
  }
  return nkt;
}

// End of the scale group of a tile that starts at k-step kb; a 256-row tile
// (a CTA pair's) ends one where either 128-row half's group ends.
__device__ __forceinline__ int64_t group_end_tile(const TileView& T, int64_t kb, int64_t nkt) {
  const int64_t e = group_end(T.gmask, kb, nkt);
  return T.gmask2 ? min(e, group_end(T.gmask2, kb, nkt)) : e;
}

// MMA N of a tile: its boxes are 64 columns wide, but when the last one is a
// checksum box (bsplit < nbox) only its columns below the checksum width C16
// are used, so N stops at the first multiple of 16 past them.  The TMEM columns
// beyond N are never stored (checksum columns >= C16) and no fused sum reads
// checksum columns.
__device__ __forceinline__ int mma_cols(int nbox, int bsplit, int64_t colC, int64_t C16) {
  if (bsplit >= nbox) return 64 * nbox;
  const int64_t first = colC + 64 * (nbox - 1 - bsplit);  // first column of the last box
  const int64_t used = C16 - first < 64 ? C16 - first : 64;
  return 64 * (nbox - 1) + (used > 0 ? (int)((used + 15) / 16 * 16) : 64);
}

// One problem (abft_gemm), tiles of kBM rows (128 or 256).
template <int kBM>
struct SingleSched {
  const TcMaps* M;
  const TcArgs* a;
  __device__ __forceinline__ int64_t total() const { return a->t_total; }
  __device__ __forceinline__ void prefetch() const {
    for (int pl = 0; pl < kPlanes; ++pl) {
      tc::prefetch_tmap(&M->a[pl]);
      tc::prefetch_tmap(&M->acs[pl]);
      tc::prefetch_tmap(&M->b[pl]);
      tc::prefetch_tmap(&M->bcs[pl]);
      tc::prefetch_tmap(&M->a128[pl]);
      tc::prefetch_tmap(&M->b4[pl]);
    }
  }
  __device__ __forceinline__ TileView view(int64_t t) const {
    const TcArgs& g = *a;
    const Tile T = g.f8 ? decode_cs_spread(t, g.ntm, g.ntn, g.ntr, g.ntc, g.group_m, kBM,
                                           g.cs_stride)
                        : decode_local(t, g.ntm, g.ntn, g.ntr, g.ntc, g.group_m, kBM);
    TileView V;
    V.prob = 0;
    V.nkb = (g.k + BK - 1) / BK;
    V.nseg = g.nseg;
    V.kpg = g.kpg;
    V.seg_a = g.seg_a;
    V.seg_b = g.seg_b;
    V.maD = &M->a[0];
    V.maC = &M->acs[0];
    V.mbD = &M->b[0];
    V.mbC = &M->bcs[0];
    V.rowD = V.rowC = (int32_t)T.row0;
    V.colD = V.colC = (int32_t)T.col0;
    const int hrows =
        (int)clamp64(cdiv((T.kind == 1 ? g.R16 : g.m) - T.row0, 64), 1, kBM / 64);
    const int bcols = (int)clamp64(cdiv((T.kind == 2 ? g.C16 : g.n) - T.col0, 64), 1, 4);
    V.hsplit = T.kind == 1 ? 0 : hrows;
    V.hcnt = hrows;
    V.bsplit = T.kind == 2 ? 0 : bcols;
    V.nbox = bcols;
    V.nmma = mma_cols(V.nbox, V.bsplit, T.col0, g.C16);
    V.swap = V.nsw_h = V.nsw_n = 0;
    V.k2 = 1;
    V.maW = V.mbW = nullptr;
    V.rowW = (int32_t)T.row0;
    V.colW = (int32_t)T.col0;
    V.nA128 = hrows % 2 == 0 ? hrows / 2 : 0;  // whole 128-row boxes, else per half
    if (V.nA128) V.maW = T.kind == 1 ? &M->acs128[0] : &M->a128[0];
    V.nW = 4;
    if (bcols == 4 && T.col0 + 256 <= ((T.kind == 2 ? g.C16 : g.n) / 64) * 64) {
      V.mbW = T.kind == 2 ? &M->bcs4[0] : &M->b4[0];
    }
    V.f8 = g.f8 && T.kind == 0;
    V.sArow = nullptr;
    V.sB = g.sB;
    V.nsb = g.nsb;
    V.gmask = nullptr;
    V.sArow2 = nullptr;
    V.gmask2 = nullptr;
    if (V.f8) {  // data tile on the e4m3 codes: 128-wide k-steps in scale groups
      V.nkb = (g.k + 127) / 128;
      V.nseg = 1;
      V.kpg = 0;
      V.gmask = g.f8grp + ((T.row0 / 128) * g.ntn + T.col0 / 256) * g.f8words;
      V.seg_a = V.seg_b = 0;
      V.maD = &M->a[kF8Slot];
      V.mbD = &M->b[kF8Slot];
      V.maW = V.nA128 ? &M->a128[kF8Slot] : nullptr;
      V.mbW = (bcols == 4 && T.col0 + 256 <= g.n) ? &M->b4[kF8Slot] : nullptr;
      V.sArow = g.sA + (T.row0 / 128) * g.nsa;
      if (kBM == 256 && T.row0 + 128 < g.m) {
        V.sArow2 = V.sArow + g.nsa;
        V.gmask2 = V.gmask + g.ntn * g.f8words;
      }
    }
    V.C = g.C;
    V.ldc = g.ldc;
    V.m = g.m;
    V.n = g.n;
    V.E16 = g.E16;
    V.R16 = g.R16;
    V.F16 = g.F16;
    V.C16 = g.C16;
    V.sC = (g.st_ok & 1) ? &M->cst : nullptr;
    V.sE = (g.st_ok & 2) ? &M->est : nullptr;
    V.sF = (g.st_ok & 4) ? &M->fst : nullptr;
    V.obs_col = T.kind == 0 ? g.obs_col : nullptr;
    V.obs_row = g.obs_row;
    V.g = g.g;
    V.ngrp = g.ngrp;
    V.vb_r = g.vb_r;
    V.vb_c = g.vb_c;
    V.er = g.er;
    V.ec = g.ec;
    return V;
  }
};

// Row-wise store of one lane's 32 consecutive values (lane = row), for
// outputs without a TMA store map (a leading dimension or base address that
// is not 16-byte aligned).
__device__ __forceinline__ void store_row32(float* dst, int64_t ld, int64_t row, int64_t col,
                                            int64_t clim, const float (&v)[32]) {
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

// One warp's 32 x 32 fp32 staging block for the TMA store of a chunk: row r
// (128 bytes) at r * 128, its 16-byte unit j at unit j ^ (r % 8) -- the
// 128-byte swizzle of a TMA box with 32 fp32 columns (the block is
// 1024-byte aligned).  Lane r writes its row: for each unit the 32 lanes
// cover all 32 banks once per 8 rows (4 wavefronts, the minimum).
__device__ __forceinline__ void stage_row32(float* stg, int lane, const float (&v)[32]) {
  float4* rowp = reinterpret_cast<float4*>(stg + lane * 32);
#pragma unroll
  for (int j = 0; j < 8; ++j)
    rowp[j ^ (lane & 7)] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
}

// The kernel body, shared by the single-problem and the grouped product.
// kPromote: the K loop runs in promotion groups whose accumulators the
// epilogue sums in fp32 registers (a separate instantiation, so the register
// accumulator of that path does not weigh on the single-group epilogue).
// kPair: 256 x 256 tiles on a CTA pair (see Geo); this CTA takes rows
// 128 rank .. of every tile, the even CTA issues the MMAs for both.
template <bool kPromote, bool kTall, bool kF8, bool kPair, class Sched>
__device__ __forceinline__ void tc_body(const Sched& S, int* status, uint64_t wait_ns,
                                        int stall_test, const int32_t* inj_hdr,
                                        const InjectEntry* inj) {
  using G = Geo<kTall, kPair>;
  static_assert(!(kPromote && kTall), "promotion runs on regular or pair tiles");
  static_assert(!kF8 || kPromote, "FP8 data tiles promote every k-step");
  static_assert(!kTall || kEpiWarps == 8, "tall tiles: one epilogue warp per lane quarter and half");
  constexpr int NS = G::kStages;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint64_t* bars =
      reinterpret_cast<uint64_t*>(smem + NS * G::kStageBytes + kEpiWarps * STG_BYTES);
  // bars[0..S): full, [S..2S): empty, [2S..2S+2): tmem full, [2S+2..2S+4): tmem empty,
  // [2S+4]: drain
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * NS + 5);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto full = [&](int s) { return tc::smem_addr(&bars[s]); };
  auto empty = [&](int s) { return tc::smem_addr(&bars[NS + s]); };
  auto tfull = [&](int a) { return tc::smem_addr(&bars[2 * NS + a]); };
  auto tempty = [&](int a) { return tc::smem_addr(&bars[2 * NS + 2 + a]); };
  const uint32_t drain = tc::smem_addr(&bars[2 * NS + 4]);
  // CTA pair: this CTA's rank; the MMA issuer's (even CTA's) stage-full and
  // accumulator-empty barriers count both CTAs' bytes and epilogue warps
  const uint32_t rank = kPair ? tc::cluster_ctarank() : 0u;
  const bool issuer = rank == 0;
  auto full_i = [&](int s) { return kPair ? tc::mapa(full(s), 0) : full(s); };
  auto tempty_i = [&](int a) { return kPair ? tc::mapa(tempty(a), 0) : tempty(a); };
  // persistent tile loop: tiles per CTA (per pair)
  const int64_t tfirst = kPair ? (int64_t)tc::cluster_id() : (int64_t)blockIdx.x;
  const int64_t tstep = kPair ? (int64_t)tc::num_clusters() : (int64_t)gridDim.x;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      tc::mbar_init(full(s), 2);  // the A and the B producer each arrive with their bytes
      tc::mbar_init(empty(s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      tc::mbar_init(tfull(a), 1);
      tc::mbar_init(tempty(a), kPair ? 2 * kEpiWarps : kEpiWarps);
    }
    tc::mbar_init(drain, 1);
    *abort = 0;
    tc::wait_limit_ns() = wait_ns;
    tc::fence_barrier_init();
    S.prefetch();
  }
  if (warp == 1) {
    if constexpr (kPair) {  // one warp of each CTA, together
      tc::tmem_alloc_pair(tc::smem_addr(tmem_slot), TMEM_COLS);
      tc::tmem_relinquish_pair();
    } else {
      tc::tmem_alloc(tc::smem_addr(tmem_slot), TMEM_COLS);
      tc::tmem_relinquish();
    }
  }
  tc::fence_before_sync();
  if constexpr (kPair)
    tc::cluster_sync();  // the peer's barriers are initialised before any use
  else
    __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const int64_t total = S.total();

  if (warp == 0 || warp == kWarpProdB) {
    if (lane == 0) {
      // ---------------- TMA producers: warp 0 copies A, warp kWarpProdB copies
      // B (two issuing threads: one thread's issue rate limited the ring);
      // each arrives on the stage's full barrier with its own bytes
      const bool pA = warp == 0;
      int s = 0;
      uint32_t ph = 0;
      int64_t issued = 0;  // stages filled and not known to be consumed
      for (int64_t t = tfirst; t < total && !*abort; t += tstep) {
        const TileView T = S.view(t);
        if (stall_test && t == 0) continue;  // nothing will fill these stages
        const int64_t nkb = T.nkb, nkt = T.nkb * T.nseg;
        if constexpr (!kPair && !kTall && !kF8) {
          if (T.k2 == 2) {
            // checksum-column tile (grouped, one plane): two k-steps per stage,
            // the second k-step's A in the first 16 KiB of the B region and the
            // checksum box of k-step j at 16 + 8 j KiB of it
            for (int64_t kb = 0; kb < nkb && !*abort; kb += 2) {
              const int kbs = nkb - kb >= 2 ? 2 : 1;
              if (!tc::wait(empty(s), ph ^ 1, abort)) break;
              const uint32_t sa = tc::smem_addr(smem + s * G::kStageBytes);
              tc::mbar_arrive_expect_tx(
                  full(s), (uint32_t)kbs * (pA ? (uint32_t)T.hcnt * HALF_BYTES
                                               : (uint32_t)T.nbox * B_BOX_BYTES));
              for (int j = 0; j < kbs; ++j) {
                const int32_t kx = (int32_t)((kb + j) * BK);
                if (pA) {
                  const uint32_t da = sa + (j ? G::kABytes : 0u);
                  if (T.maW) {
                    tc::tma_load_2d(da, T.maW, full(s), kx, T.rowW);
                  } else {
                    for (int h = 0; h < T.hcnt; ++h) {
                      const bool dat = h < T.hsplit;
                      tc::tma_load_2d(da + h * HALF_BYTES, dat ? T.maD : T.maC, full(s), kx,
                                      dat ? T.rowD + 64 * h : T.rowC + 64 * (h - T.hsplit));
                    }
                  }
                } else {
                  tc::tma_load_2d(sa + G::kABytes + 2 * HALF_BYTES + j * B_BOX_BYTES, T.mbC,
                                  full(s), T.colC, kx);
                }
              }
              ++issued;
              if (++s == NS) { s = 0; ph ^= 1; }
            }
            continue;
          }
        }
        // an FP8 data tile's k-step is 128 codes (128 bytes, as a bf16 k-step);
        // its B boxes hold 64 rows of B^T (8 KiB, as a bf16 box).  A pair's
        // bytes (both CTAs') land on the issuer's barrier, which the issuer's
        // producers expect: the same totals as one CTA's 256-row tile.
        const uint32_t tx = T.swap ? (pA ? (uint32_t)T.nsw_h * HALF_BYTES : 4 * B_BOX_BYTES)
                                   : pA ? (uint32_t)T.hcnt * HALF_BYTES
                                        : (uint32_t)T.nbox * B_BOX_BYTES;
        const int bkx = T.f8 ? BK8 : BK;
        // this CTA's halves [h_lo, h_hi) and boxes [b_lo, b_hi) of the tile
        // (a pair splits both: rows 128 rank .., columns 128 rank ..)
        const int h_lo = kPair ? 2 * (int)rank : 0, b_lo = kPair ? 2 * (int)rank : 0;
        const int h_hi = kPair ? min(T.hcnt, h_lo + 2) : T.hcnt;
        const int b_hi = kPair ? min(T.nbox, b_lo + 2) : T.nbox;
        // a stage's MMAs take ~700 cycles: the per-stage bookkeeping is
        // incremental (no division per stage)
        int seg = 0, pa = (int)(T.seg_a & 3u), pb = (int)(T.seg_b & 3u);
        int64_t kb = 0;
        for (int64_t kt = 0; kt < nkt; ++kt) {
          const int32_t kx = (int32_t)(kb * bkx);
          if (!tc::wait(empty(s), ph ^ 1, abort)) break;
          const uint32_t sa = tc::smem_addr(smem + s * G::kStageBytes);
          const uint32_t fb = full_i(s);
          if (issuer) tc::mbar_arrive_expect_tx(full(s), tx);
          auto load2 = [&](uint32_t dst, const CUtensorMap* map, int32_t x, int32_t y) {
            if constexpr (kPair)
              tc::tma_load_2d_pair(dst, map, fb, x, y);
            else
              tc::tma_load_2d(dst, map, fb, x, y);
          };
          if (!kPair && T.swap) {
            // swapped checksum-row tile: the A region takes the checksum rows'
            // halves (the N side), the B region four B boxes (the M side)
            if (pA) {
              for (int h = 0; h < T.nsw_h; ++h)
                tc::tma_load_2d(sa + h * HALF_BYTES, T.maC, full(s), kx, 64 * h);
            } else if (T.mbW) {
              tc::tma_load_3d(sa + G::kABytes, T.mbW, full(s), 0, kx, T.colW / 64);
            } else {
              for (int b = 0; b < 4; ++b)
                tc::tma_load_2d(sa + G::kABytes + b * B_BOX_BYTES, T.mbD, full(s), T.colW + 64 * b,
                                kx);
            }
          } else if (!pA && T.f8) {
            // e4m3 B^T (K-major): this CTA's rows of a full tile in one copy
            // (256 rows, a pair's CTA 128), else 64 rows per box
            if (T.mbW) {
              load2(sa + G::kABytes, T.mbW, kx, T.colW + 64 * b_lo);
            } else {
              for (int b = b_lo; b < b_hi; ++b)
                load2(sa + G::kABytes + (b - b_lo) * B_BOX_BYTES, T.mbD, kx, T.colD + 64 * b);
            }
          } else if (!pA) {
            // B: the full boxes in one 3-D copy (4 boxes, a pair's CTA 2), the
            // rest (ragged, checksum) per box
            int b_first = b_lo;
            if (T.mbW) {
              if constexpr (kPair)
                tc::tma_load_3d_pair(sa + G::kABytes, T.mbW + pb, fb, 0, kx, T.colW / 64 + b_lo);
              else
                tc::tma_load_3d(sa + G::kABytes, T.mbW + pb, fb, 0, kx, T.colW / 64);
              b_first = kPair ? b_hi : T.nW;  // a pair tile's W copy is all of its boxes
            }
            for (int b = b_first; b < b_hi; ++b) {
              const bool dat = b < T.bsplit;
              const CUtensorMap* mb = (dat ? T.mbD : T.mbC) + pb;
              const int32_t x = dat ? T.colD + 64 * b : T.colC + 64 * (b - T.bsplit);
              load2(sa + G::kABytes + (b - b_lo) * B_BOX_BYTES, mb, x, kx);
            }
          } else if (T.maW) {
            // whole 128-row boxes: box i at rows rowW + 128 i (a pair's CTA: box rank)
            const int i_lo = kPair ? (int)rank : 0, i_hi = kPair ? min(T.nA128, i_lo + 1) : T.nA128;
            for (int i = i_lo; i < i_hi; ++i)
              load2(sa + (i - i_lo) * (2 * HALF_BYTES), T.maW + pa, kx, T.rowW + 128 * i);
          } else {
            for (int h = h_lo; h < h_hi; ++h) {
              const bool dat = h < T.hsplit;
              const CUtensorMap* ma = (dat ? T.maD : T.maC) + pa;
              const int32_t y = dat ? T.rowD + 64 * h : T.rowC + 64 * (h - T.hsplit);
              load2(sa + (h - h_lo) * HALF_BYTES, ma, kx, y);
            }
          }
          ++issued;
          if (++s == NS) { s = 0; ph ^= 1; }
          if (++kb == nkb) {  // next K segment: its planes of A and B
            kb = 0;
            ++seg;
            pa = (int)((T.seg_a >> (2 * seg)) & 3u);
            pb = (int)((T.seg_b >> (2 * seg)) & 3u);
          }
        }
      }
      // Do not leave copies in flight: wait for the last fills (bounded).  A
      // pair's copies complete on the issuer's barriers, so its CTAs wait
      // until the MMAs consumed the stages instead (the commit that frees a
      // stage reaches both CTAs; once it arrived no signal to this CTA's
      // barriers is outstanding).
      for (int q = 0; q < NS && issued > 0; ++q, --issued) {
        if (--s < 0) { s = NS - 1; ph ^= 1; }
        const uint64_t t0 = tc::globaltimer();
        const uint32_t bar = kPair ? empty(s) : full(s);
        while (!tc::mbar_try_wait(bar, ph) && tc::globaltimer() - t0 < tc::wait_limit_ns()) {
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0 && issuer) {
      // ---------------- MMA issuer (a pair: the even CTA's, for both)
      int s = 0, acc = 0;
      uint32_t ph = 0, aph = 0;
      for (int64_t t = tfirst; t < total && !*abort; t += tstep) {
        const TileView T = S.view(t);
        const int64_t nkt = T.nkb * T.nseg;
        const int64_t gsz = (kPromote && T.kpg > 0 && T.kpg < nkt) ? T.kpg : nkt;
        const bool f8t = kF8 && T.f8;
        // a pair's MMA: M = 256 (128 rows per CTA), N = 256 (128 columns of B
        // per CTA; boxes a tile does not have are never stored)
        const int mm = kPair ? 256 : BM, nn = kPair ? BN : T.nmma;
        const uint32_t idesc = f8t ? tc::idesc_e4m3(mm, nn, 0) : tc::idesc_bf16(mm, nn, 1);
        if constexpr (!kPair && !kTall && !kF8) {
          if (T.k2 == 2) {  // checksum-column tile: two k-steps per stage (see the producers)
            if (!tc::wait(tempty(acc), aph ^ 1, abort)) break;
            tc::fence_after_sync();
            const uint32_t d = tmem + acc * BN;
            bool ok2 = true;
            for (int64_t kb = 0; kb < T.nkb; kb += 2) {
              const int kbs = T.nkb - kb >= 2 ? 2 : 1;
              if (!tc::wait(full(s), ph, abort)) { ok2 = false; break; }
              tc::fence_after_sync();
              const uint32_t sa = tc::smem_addr(smem + s * G::kStageBytes);
              for (int j = 0; j < kbs; ++j) {
                const uint32_t a0 = sa + (j ? G::kABytes : 0u);
                const uint32_t b0 = sa + G::kABytes + 2 * HALF_BYTES + j * B_BOX_BYTES;
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk)
                  tc::mma_f16_x<kPair>(d, tc::sdesc_sw128(a0 + kk * 32, 16, 1024),
                                       tc::sdesc_sw128(b0 + kk * 2048, B_BOX_BYTES, 1024), idesc,
                                       (kb > 0 || j > 0 || kk > 0) ? 1u : 0u);
              }
              tc::commit_x<kPair>(empty(s));
              if (++s == NS) { s = 0; ph ^= 1; }
            }
            if (!ok2) break;
            tc::commit_x<kPair>(tfull(acc));
            if (++acc == G::kSlots) { acc = 0; aph ^= 1; }
            continue;
          }
        }
        bool ok = true;
        // one accumulator per promotion group (FP8 data tiles: per scale
        // group); the epilogue adds the groups
        int64_t g1 = 0;
        for (int64_t g0 = 0; g0 < nkt && ok; g0 = g1) {
          g1 = f8t ? group_end_tile(T, g0, nkt) : min(g0 + gsz, nkt);
          if (!tc::wait(tempty(acc), aph ^ 1, abort)) { ok = false; break; }
          tc::fence_after_sync();
          const uint32_t d = tmem + acc * BN;
          // tall tiles: the second 128-row half only when it holds rows
          const int nmma = kTall && T.hcnt > 2 ? 2 : 1;
          for (int64_t kb = g0; kb < g1; ++kb) {
            if (!tc::wait(full(s), ph, abort)) { ok = false; break; }
            tc::fence_after_sync();
            const uint32_t sa = tc::smem_addr(smem + s * G::kStageBytes);
            const uint32_t sb = sa + G::kABytes;
            if (!kPair && T.swap) {
              // swapped tile: two MMAs per K step, MN-major A = two B boxes each
              // (64-column atoms 8 KiB apart, 8-row K groups 1024 B apart, a K
              // step of 16 rows moves 2 KiB) into accumulator columns 0 and
              // 128, K-major B = the checksum rows in the A region
              const uint32_t idesc_sw = tc::idesc_bf16_mn_a(BM, T.nsw_n);
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk) {
                const uint64_t bd = tc::sdesc_sw128(sa + kk * 32, 16, 1024);
                for (int h2 = 0; h2 < 2; ++h2) {
                  const uint64_t ad =
                      tc::sdesc_sw128(sb + h2 * (2 * B_BOX_BYTES) + kk * 2048, B_BOX_BYTES, 1024);
                  tc::mma_f16_x<kPair>(d + h2 * 128, ad, bd, idesc_sw,
                                       (kb > g0 || kk > 0) ? 1u : 0u);
                }
              }
              tc::commit_x<kPair>(empty(s));
              if (++s == NS) { s = 0; ph ^= 1; }
              continue;
            }
            if (f8t) {
              // e4m3: K = 32 codes per MMA.  A and B^T: K-major 128-byte rows in
              // 8-row groups 1024 B apart; a K step moves 32 B inside the
              // swizzled rows.
#pragma unroll
              for (int kk = 0; kk < BK8 / 32; ++kk) {
                const uint64_t bd = tc::sdesc_sw128(sb + kk * 32, 16, 1024);
                const uint64_t ad = tc::sdesc_sw128(sa + kk * 32, 16, 1024);
                tc::mma_f8_x<kPair>(d, ad, bd, idesc, (kb > g0 || kk > 0) ? 1u : 0u);
              }
              tc::commit_x<kPair>(empty(s));
              if (++s == NS) { s = 0; ph ^= 1; }
              continue;
            }
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
              // B: N-major, 64-column boxes 8 KiB apart, 8-row (K) groups
              // 1024 B apart; a K step of 16 rows moves 2 KiB.
              const uint64_t bd = tc::sdesc_sw128(sb + kk * 2048, B_BOX_BYTES, 1024);
              for (int h2 = 0; h2 < nmma; ++h2) {
                // A: K-major, 128-byte rows, 8-row groups 1024 B apart; a K
                // step of 16 elements moves 32 B inside the swizzled row; the
                // second 128-row half starts 16 KiB later and accumulates into
                // the second TMEM accumulator
                const uint64_t ad = tc::sdesc_sw128(sa + h2 * (2 * HALF_BYTES) + kk * 32, 16, 1024);
                tc::mma_f16_x<kPair>(d + h2 * BN, ad, bd, idesc, (kb > g0 || kk > 0) ? 1u : 0u);
              }
            }
            tc::commit_x<kPair>(empty(s));
            if (++s == NS) { s = 0; ph ^= 1; }
          }
          if (!ok) break;
          tc::commit_x<kPair>(tfull(acc));
          if (++acc == G::kSlots) { acc = 0; aph ^= 1; }
        }
        if (!ok) break;
      }
      // Every MMA issued so far must complete before TMEM is freed.
      if constexpr (kPair)
        tc::commit_pair(drain, 1);
      else
        tc::commit(drain);
      const uint64_t t0 = tc::globaltimer();
      while (!tc::mbar_try_wait(drain, 0) && tc::globaltimer() - t0 < tc::wait_limit_ns()) {
      }
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: warps 2..9; TMEM lane quarter q = warp % 4 (a
    // warp may only read its quarter), column half = (warp - 2) / 4.  Each
    // 32 x 32 chunk goes to this warp's staging block in shared memory (the
    // 128-byte-swizzled layout of a TMA box) and from there to global memory
    // by a TMA store; the fused column sums read the staged columns back.
    // regular tiles: warp (w - 2) / 4 takes one 128-column half of the tile;
    // tall tiles: it takes the accumulator of 128-row half (w - 2) / 4, all
    // 256 columns
    // pair tiles: this CTA's rows are the tile's halves 2 rank, 2 rank + 1
    const int q = warp & 3, ta = kTall ? (warp - 2) >> 2 : 0;
    const int half = 2 * (kPair ? (int)rank : ta) + (q >> 1);  // this warp's 64-row half of the tile
    const int c_lo = kTall ? 0 : kEpiCols * ((warp - 2) >> 2);
    float* stg = reinterpret_cast<float*>(smem + NS * G::kStageBytes + (warp - 2) * STG_BYTES);
    const uint32_t stg_addr = tc::smem_addr(stg);
    const int ninj = (inj_hdr && inj_hdr[0] == kInjectMagic)
                         ? max(0, min(inj_hdr[1], kMaxInject)) : 0;
    int acc = 0;
    uint32_t aph = 0;
    bool aborted = false;
    // an accumulator is free again once every epilogue warp (of both CTAs of
    // a pair) has read it
    auto release = [&](int a) {
      if constexpr (kPair)
        tc::mbar_arrive_cluster(tempty_i(a));
      else
        tc::mbar_arrive(tempty(a));
    };
    for (int64_t t = tfirst; t < total && !aborted; t += tstep) {
      const TileView T = S.view(t);
      if (T.swap) {
        // swapped checksum-row tile: this warp's half h of the tile (columns
        // colW + 128 h ..) sits in accumulator columns 128 h .., TMEM lane
        // quarter q holds columns + 32 q .., lane = column j of E16 and
        // accumulator column 128 h + r = checksum row r; each store instruction
        // writes one row r for 32 consecutive columns
        if (!tc::wait(tfull(acc), aph, abort)) break;
        tc::fence_after_sync();
        const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + acc * BN + c_lo;
        const int nchs = (T.nsw_n + 31) / 32;
        const int64_t j = T.colW + c_lo + 32 * q + lane;
        for (int ci = 0; ci < nchs; ++ci) {
          float v[32];
          tc::tmem_ld32(base + 32 * ci, v);
          if (ci == nchs - 1) {
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) release(acc);
            if (++acc == G::kSlots) { acc = 0; aph ^= 1; }
          }
          if (j < T.n) {
#pragma unroll
            for (int u = 0; u < 32; ++u) {
              const int64_t r = 32 * ci + u;
              if (r < T.R16) T.E16[r * T.n + j] = v[u];
            }
          }
        }
        if (nchs <= 0) {
          tc::fence_before_sync();
          __syncwarp();
          if (lane == 0) release(acc);
          if (++acc == G::kSlots) { acc = 0; aph ^= 1; }
        }
        continue;
      }
      const int64_t nkt = T.nkb * T.nseg;
      const int64_t gsz = (kPromote && T.kpg > 0 && T.kpg < nkt) ? T.kpg : nkt;
      const bool f8t = kF8 && T.f8;
      const bool one_group = f8t ? group_end_tile(T, 0, nkt) >= nkt : gsz >= nkt;
      // FP8 data tiles: this warp's 128 columns are one column block of B's
      // scales; the partial of a scale group is multiplied by its (power-of-two,
      // so exact) block-scale product.  This CTA's row block: a pair's odd CTA
      // takes the tile's second one (none past the data: nothing is stored)
      const int64_t jb = f8t ? (T.colD + c_lo) / 128 : 0;
      const float* sArow = (kPair && rank) ? T.sArow2 : T.sArow;
      auto f8scale = [&](int64_t kb) {
        return __ldg(&sArow[kb]) * __ldg(&T.sB[kb * T.nsb + jb]);
      };
      const int ncol = 64 * T.nbox;
      const int c_hi = min(c_lo + G::kCols, ncol);
      // this warp's 32 rows: data rows, checksum rows or none
      const bool drow = half < T.hsplit, crow = !drow && half < T.hcnt;
      const int64_t rin = 32 * (q & 1) + lane;
      const int64_t row = drow ? T.rowD + 64 * half + rin : T.rowC + 64 * (half - T.hsplit) + rin;
      const int64_t r0 = row - lane;  // first of the warp's 32 rows
      const bool rvalid = drow ? row < T.m : (crow && row < T.R16);
      const int ndcol = 64 * T.bsplit;
      const bool fused = T.obs_col != nullptr && T.hsplit > 0 && T.bsplit > 0;
      // armed faults inside this warp's part of the tile (one pass over the list)
      bool inj_hit = false;
      if (drow && ninj > 0) {
        const int64_t c0 = T.colD + c_lo;
        for (int f = lane; f < ninj; f += 32) {
          const InjectEntry ie = inj[f];
          inj_hit |= ie.pad == T.prob && ie.row >= r0 && ie.row < r0 + 32 && ie.col >= c0 &&
                     ie.col < c0 + G::kCols;
        }
        inj_hit = __any_sync(0xffffffffu, inj_hit);
      }
      const float scr = scalbnf(1.0f, -T.er), scc = scalbnf(1.0f, -T.ec);
      float racc_e = 0.f, racc_w = 0.f;
      // verify-block and group offsets of the warp's rows and the tile's
      // columns, once per tile (64-bit division is a software routine);
      // the chunks use 32-bit offsets from them
      const int g32 = (int)T.g;
      const int rb0 = fused ? (int)(r0 % T.vb_r) + 1 : 1;  // weight of row r0
      const int cm0 = fused ? (int)(T.colD % T.vb_c) : 0;
      const int cg0 = fused ? (int)(T.colD % T.g) : 0;
      const int64_t gi0 = fused ? T.colD / T.g : 0;
      // Column partials of this warp's 32 rows (r0 ..) for the chunk at
      // column col, from the staged block (no shuffles: each lane sums one
      // column); weights of the rows in their verify block (the 32 rows never
      // straddle one).  They run one chunk late, after the next chunk's TMEM
      // load and row partials, so the staged block is read well after its
      // writes were fenced for the TMA store.
      bool cs_pend = false;
      int64_t cs_col = 0;
      float* const obs_base = fused ? T.obs_col + (r0 >> 5) * 2 * T.n : nullptr;
      // the row partials' column position, kept incrementally: the chunks of a
      // tile come in column order, 32 apart, and the verify block width vb_c
      // and the group width g are multiples of 32 when the sums are fused
      int cm_run = fused ? (cm0 + c_lo) % T.vb_c : 0;             // (cm0 + c) % vb_c
      int cg_run = fused ? (cg0 + c_lo) % g32 : 0;                // (cg0 + c) % g
      int64_t gi_run = fused ? gi0 + (cg0 + c_lo) / g32 : 0;      // group of column colD + c
      auto colsum = [&](int64_t col) {
        // lane = column: its 32 rows of the staged block (row r's 16-byte unit
        // j at unit j ^ (r % 8): one conflict-free word per lane and row), in
        // four independent partial sums.  Row r's weight (rb0 + r) scr lies in
        // (0, 1] and is exact, so a weighted term never exceeds its element
        // (no overflow that the element itself does not have) and an infinite
        // element gives an infinite sum.
        const int u4 = lane >> 2, sub = lane & 3;
        float a[4] = {0.f, 0.f, 0.f, 0.f}, b[4] = {0.f, 0.f, 0.f, 0.f};
        float wr = (float)rb0 * scr;
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          const float x = stg[r * 32 + ((u4 ^ (r & 7)) << 2) + sub];
          a[r & 3] += x;
          b[r & 3] = fmaf(wr, x, b[r & 3]);
          wr += scr;
        }
        const int64_t c = col + lane;
        if (r0 < T.m && c < T.n) {
          obs_base[c] = (a[0] + a[1]) + (a[2] + a[3]);
          obs_base[T.n + c] = (b[0] + b[1]) + (b[2] + b[3]);
        }
      };
      auto flush = [&]() {
        if (cs_pend) {
          cs_pend = false;
          colsum(cs_col);
        }
      };
      // Stage v (lane = row) into this warp's block; with a store map, send
      // the block to (x, y) by one TMA store.  The block is reused only after
      // the pending column partials have read it, the previous store has
      // read it and every lane is past its reads.
      auto stage = [&](const float (&v)[32], const CUtensorMap* map, int64_t x, int64_t y) {
        flush();
        if (lane == 0) tc::bulk_wait_read0();
        __syncwarp();
        stage_row32(stg, lane, v);
        if (map) tc::fence_proxy_async_smem();
        __syncwarp();
        if (map && lane == 0) {
          tc::tma_store_2d(map, stg_addr, (int32_t)x, (int32_t)y);
          tc::bulk_commit();
        }
      };
      // one 32-column chunk of the finished tile: fault injection, row
      // partials (lane = row), store, column partials (v is consumed)
      auto chunk = [&](int c, float (&v)[32]) {
        const bool dcol = c < ndcol;
        if (dcol) {
          const int64_t col = T.colD + c;
          if (col >= T.n) return;
          if (drow && inj_hit)
            for (int f = 0; f < ninj; ++f) {
              const InjectEntry ie = inj[f];
              if (ie.pad == T.prob && ie.row == row && ie.col >= col && ie.col < col + 32) {
                const int x = ie.col - (int)col;
#pragma unroll
                for (int u = 0; u < 32; ++u)
                  if (u == x) v[u] = __uint_as_float(__float_as_uint(v[u]) ^ (1u << (ie.bit & 31)));
              }
            }
          if (fused && drow) {
            // row partials over the column group (weights restart per verify
            // block; a 32-column chunk never straddles one, a group never
            // straddles the two column halves): sum_u (cm + u) scc v[u] as
            // scc (cm sum_u v[u] + sum_u u v[u])
            // four independent partial sums each (short dependency chains);
            // s1 weighs v[u] by u / 32 < 1, so no weighted term exceeds its
            // element, and sum_u (cm + u) scc v[u] = cm scc s0 + 32 scc s1
            float a[4] = {0.f, 0.f, 0.f, 0.f}, b[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int u = 0; u < 32; u += 4) {
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                a[j] += v[u + j];
                b[j] = fmaf((float)(u + j) * 0.03125f, v[u + j], b[j]);
              }
            }
            const float s0 = (a[0] + a[1]) + (a[2] + a[3]);
            const float s1 = (b[0] + b[1]) + (b[2] + b[3]);
            racc_e += s0;
            racc_w = fmaf((float)(cm_run + 1) * scc, s0, fmaf(32.0f * scc, s1, racc_w));
            if (cg_run + 32 == g32 || c + 32 == ndcol || col + 32 >= T.n) {
              if (rvalid) {
                float* o = T.obs_row + (row * T.ngrp + gi_run) * 2;
                o[0] = racc_e;
                o[1] = racc_w;
              }
              racc_e = racc_w = 0.f;
            }
            cm_run += 32;
            if (cm_run >= T.vb_c) cm_run -= T.vb_c;
            cg_run += 32;
            if (cg_run >= g32) {
              cg_run -= g32;
              ++gi_run;
            }
          }
          if (!drow && !crow) return;
          if (r0 >= (drow ? T.m : T.R16)) return;  // all 32 rows past the output
          const CUtensorMap* map = drow ? T.sC : T.sE;
          const bool colsums = fused && drow;
          if (map || colsums) stage(v, map, col, r0);
          if (!map && rvalid) store_row32(drow ? T.C : T.E16, drow ? T.ldc : T.n, row, col, T.n, v);
          if (colsums) {
            if constexpr (kPromote) {
              colsum(col);  // the promoted epilogue has no registers to spare
            } else {        // read back from the staged block one chunk later
              cs_pend = true;
              cs_col = col;
            }
          }
        } else if (drow && r0 < T.m) {
          const int64_t col = T.colC + (c - ndcol);
          if (col < T.C16) {
            if (T.sF)
              stage(v, T.sF, col, r0);
            else if (rvalid)
              store_row32(T.F16, T.C16, row, col, T.C16, v);
          }
        }
      };
      if (!kPromote || one_group) {
        // one accumulator: each chunk is read and finished in turn; the
        // accumulator is released after the last read
        if (!tc::wait(tfull(acc), aph, abort)) break;
        tc::fence_after_sync();
        const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + (acc + ta) * BN;
        const int nch = (c_hi - c_lo + 31) / 32;
        const float sc1 = (f8t && nch > 0 && sArow) ? f8scale(0) : 1.0f;
        for (int ci = 0; ci < nch; ++ci) {
          float v[32];
          tc::tmem_ld32(base + c_lo + 32 * ci, v);
          if (f8t) {
#pragma unroll
            for (int u = 0; u < 32; ++u) v[u] *= sc1;
          }
          if (ci == nch - 1) {
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) release(acc);
            if (++acc == G::kSlots) { acc = 0; aph ^= 1; }
          }
          chunk(c_lo + 32 * ci, v);
        }
        flush();
        if (nch <= 0) {  // nothing of this tile in this warp's half
          tc::fence_before_sync();
          __syncwarp();
          if (lane == 0) release(acc);
          if (++acc == G::kSlots) { acc = 0; aph ^= 1; }
        }
      } else if constexpr (kPromote) {
        // promotion groups: this warp's part of the tile summed over the
        // groups in fp32 registers (round to nearest), each accumulator
        // released as soon as it is read
        float accr[kEpiChunks][32];
        // FP8 data tiles: each scale group's partial times its block scales;
        // the next group's scale is loaded ahead
        const bool scaled = f8t && c_lo < c_hi && sArow;
        float sc_next = scaled ? f8scale(0) : 1.0f;
        int64_t g1 = 0;
        for (int64_t g0 = 0; g0 < nkt; g0 = g1) {
          g1 = f8t ? group_end_tile(T, g0, nkt) : min(g0 + gsz, nkt);
          const float sc = sc_next;
          if (scaled && g1 < nkt) sc_next = f8scale(g1);
          if (!tc::wait(tfull(acc), aph, abort)) { aborted = true; break; }
          tc::fence_after_sync();
          const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + acc * BN;
#pragma unroll
          for (int ci = 0; ci < kEpiChunks; ++ci) {
            const int c = c_lo + 32 * ci;
            if (c < c_hi) {
              if (g0 == 0) {
                tc::tmem_ld32(base + c, accr[ci]);
                if (scaled) {
#pragma unroll
                  for (int u = 0; u < 32; ++u) accr[ci][u] *= sc;
                }
              } else {
                float v[32];
                tc::tmem_ld32(base + c, v);
                if (scaled) {
#pragma unroll
                  for (int u = 0; u < 32; ++u) accr[ci][u] = fmaf(sc, v[u], accr[ci][u]);
                } else {
#pragma unroll
                  for (int u = 0; u < 32; ++u) accr[ci][u] += v[u];
                }
              }
            }
          }
          tc::fence_before_sync();
          __syncwarp();
          if (lane == 0) release(acc);
          if (++acc == 2) { acc = 0; aph ^= 1; }
        }
        if (aborted) break;
#pragma unroll
        for (int ci = 0; ci < kEpiChunks; ++ci)
          if (c_lo + 32 * ci < c_hi) chunk(c_lo + 32 * ci, accr[ci]);
        flush();
      }
    }
    // every TMA store of this warp has completed before the kernel ends
    if (lane == 0) tc::bulk_wait0();
    __syncwarp();
  }


  tc::fence_before_sync();
  // a pair: neither CTA frees TMEM or exits while the other may still signal
  // its barriers or (the issuer's MMAs) read its shared memory
  if constexpr (kPair)
    tc::cluster_sync();
  else
    __syncthreads();
  if (threadIdx.x == 0 && *abort) atomicExch(status, 1);
  if (warp == 1) {
    tc::fence_after_sync();
    if constexpr (kPair)
      tc::tmem_dealloc_pair(tmem, TMEM_COLS);
    else
      tc::tmem_dealloc(tmem, TMEM_COLS);
  }
  if constexpr (kPair) tc::cluster_sync();
}

template <bool kPromote, bool kTall, bool kF8, bool kPair>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_bf16(const __grid_constant__ TcMaps M, const TcArgs g) {
  const SingleSched<Geo<kTall, kPair>::kBM> S{&M, &g};
  tc_body<kPromote, kTall, kF8, kPair>(S, g.status, g.wait_ns, g.stall_test, g.inj_hdr, g.inj);
}

// Many problems (grouped product).  The flattened tile list is a table of
// (problem, tile row, tile column) entries; per-problem sizes, outputs and
// tensor maps live in global memory.  A problem's rows are its 64-row data
// halves followed by its checksum halves, its columns its 64-column data
// boxes followed by its checksum boxes, cut into tiles of two halves and
// bpt boxes, so checksum rows and columns fill the padding of the last data
// tiles.  Verify blocks are 128 rows (one tile row) x 256 columns.
struct GroupSched {
  const GProb* probs;
  const GMaps* maps;
  const int4* tiles;  // {problem, tile row, tile column, 0}
  int64_t t_total;
  bool checksums;
  int kpg;
  __device__ __forceinline__ int64_t total() const { return t_total; }
  __device__ __forceinline__ void prefetch() const {}
  __device__ __forceinline__ TileView view(int64_t t) const {
    const int4 e = __ldg(&tiles[t]);
    const GProb& P = probs[e.x];
    const GMaps& Mp = maps[e.x];
    const int nhd = (int)cdiv(P.m, 64), nbd = (int)cdiv(P.n, 64);
    const int nhc = checksums && !P.swap_rows ? P.nhc : 0, nbc = checksums ? P.nbc : 0;
    const int h0 = 2 * e.y, b0 = P.bpt * e.z;
    TileView V;
    V.prob = e.x;
    V.nkb = cdiv(P.k, BK);
    V.nseg = 1;
    V.kpg = kpg;
    V.seg_a = V.seg_b = 0;  // one plane
    V.maD = &Mp.a;
    V.maC = &Mp.acs;
    V.mbD = &Mp.b;
    V.mbC = &Mp.bcs;
    V.hsplit = max(0, min(2, nhd - h0));
    V.hcnt = min(2, nhd + nhc - h0);
    V.bsplit = max(0, min(P.bpt, nbd - b0));
    V.nbox = min(P.bpt, nbd + nbc - b0);
    V.rowD = 64 * h0;
    V.rowC = 64 * max(0, h0 - nhd);
    V.colD = 64 * b0;
    V.colC = 64 * max(0, b0 - nbd);
    V.nmma = mma_cols(V.nbox, V.bsplit, V.colC, P.C16);
    V.swap = V.nsw_h = V.nsw_n = 0;
    V.k2 = 1;
    V.maW = V.mbW = nullptr;
    V.nA128 = 1;
    if (V.hsplit == 2) {
      V.maW = &Mp.a128;
      V.rowW = V.rowD;
    } else if (V.hsplit == 0 && V.hcnt == 2) {
      V.maW = &Mp.acs128;
      V.rowW = V.rowC;
    }
    if (V.bsplit >= 2 && b0 + V.bsplit <= (int)(P.n / 64)) {  // full data boxes
      V.mbW = &Mp.bw[V.bsplit - 2];
      V.colW = V.colD;
      V.nW = V.bsplit;
    } else if (V.nbox == 4 && V.bsplit == 0 && (b0 - nbd) + 4 <= (int)(P.C16 / 64)) {
      V.mbW = &Mp.bcs4;
      V.colW = V.colC;
      V.nW = 4;
    }
    V.C = P.C;
    V.ldc = P.ldc;
    V.m = P.m;
    V.n = P.n;
    V.E16 = P.E16;
    V.R16 = P.R16;
    V.F16 = P.F16;
    V.C16 = P.C16;
    V.sC = (P.st_ok & 1) ? &Mp.cst : nullptr;
    V.sE = (P.st_ok & 2) ? &Mp.est : nullptr;
    V.sF = (P.st_ok & 4) ? &Mp.fst : nullptr;
    V.obs_col = checksums ? P.obs_col : nullptr;
    V.obs_row = P.obs_row;
    V.g = P.g;
    V.ngrp = P.ngrp;
    V.vb_r = kGrpVbR;
    V.vb_c = kGrpVbC;
    V.er = kGrpEr;
    V.ec = kGrpEc;
    V.f8 = false;
    V.sArow = nullptr;
    V.sB = nullptr;
    V.nsb = 0;
    V.gmask = nullptr;
    V.sArow2 = nullptr;
    V.gmask2 = nullptr;
    if (e.w == kGrpF2Tile) V.k2 = 2;
    if (e.w == kGrpSwapTile) {  // E16 columns 256 e.z .. + 255 from the swapped operands
      V.swap = 1;
      V.nsw_h = (int)cdiv(P.R16, 64);
      V.nsw_n = (int)cdiv(P.R16, 16) * 16;
      V.colW = 256 * e.z;
      V.mbD = &Mp.b;
      V.mbW = V.colW + 256 <= (int32_t)((P.n / 64) * 64) ? &Mp.bw[2] : nullptr;
      V.maC = &Mp.acs;
      V.hsplit = V.hcnt = V.bsplit = V.nbox = 0;
      V.obs_col = nullptr;
    }
    return V;
  }
};

__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_grouped(const GProb* probs, const GMaps* maps, const int4* tiles, int64_t t_total,
                   int checksums, int* status, uint64_t wait_ns, const int32_t* inj_hdr,
                   const InjectEntry* inj, int kpg) {
  const GroupSched S{probs, maps, tiles, t_total, checksums != 0, kpg};
  tc_body<false, false, false, false>(S, status, wait_ns, 0, inj_hdr, inj);
}

// a1 b1 == a0 b0, decided without rounding: true when the scales are the same
// bits, or when all four are normal powers of two whose products have the same
// sign and exponent; false (a group boundary) otherwise.  Exact for the power-of-
// two scales the FP8 path accepts; for any other scale it may split a run that
// did not change, which costs an accumulator switch, never a wrong scale.
__device__ __forceinline__ bool same_scale_product(float a1, float b1, float a0, float b0) {
  const uint32_t x1 = __float_as_uint(a1), y1 = __float_as_uint(b1);
  const uint32_t x0 = __float_as_uint(a0), y0 = __float_as_uint(b0);
  if (x1 == x0 && y1 == y0) return true;
  auto pow2 = [](uint32_t x) {
    const uint32_t e = (x >> 23) & 0xFFu;
    return (x & 0x7FFFFFu) == 0u && e != 0u && e != 0xFFu;
  };
  if (!(pow2(x1) && pow2(y1) && pow2(x0) && pow2(y0))) return false;
  return ((x1 ^ y1) >> 31) == ((x0 ^ y0) >> 31) &&
         ((x1 >> 23) & 0xFFu) + ((y1 >> 23) & 0xFFu) == ((x0 >> 23) & 0xFFu) + ((y0 >> 23) & 0xFFu);
}

// Scale groups of the FP8 data tiles (see TcArgs::f8grp): one warp per word
// of one tile (tile row I of 128 rows, tile column Jt of 256 columns = scale
// column blocks 2 Jt and 2 Jt + 1), integer comparisons only (GB300's FP64
// pipe made the binary64 products and conversions of an earlier version cost
// 30 us).
__global__ void k_f8_groups(const float* __restrict__ sA, const float* __restrict__ sB,
                            int64_t nsa, int64_t nsb, int64_t ntm, int64_t ntn, int64_t nkb,
                            int64_t words, uint32_t* __restrict__ out) {
  // one warp per word, lane = k-step of the word (the whole warp shares the
  // word); grid (the words of a tile row / 8 warps, tile rows up to 65535)
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;  // word within a tile row
  const int lane = threadIdx.x & 31;
  if (gw >= (uint32_t)(ntn * words)) return;
  const int64_t w = gw % (uint32_t)words, Jt = gw / (uint32_t)words;
  const int64_t J0 = 2 * Jt, J1 = 2 * Jt + 1;
  const int64_t kb = w * 32 + lane;
  for (int64_t I = blockIdx.y; I < ntm; I += gridDim.y) {
    bool diff = false;
    if (kb >= 1 && kb < nkb) {
      const float a1 = sA[I * nsa + kb], a0 = sA[I * nsa + kb - 1];
      diff = !same_scale_product(a1, sB[kb * nsb + J0], a0, sB[(kb - 1) * nsb + J0]);
      if (J1 < nsb)
        diff |= !same_scale_product(a1, sB[kb * nsb + J1], a0, sB[(kb - 1) * nsb + J1]);
    }
    const uint32_t bits = __ballot_sync(0xffffffffu, diff);
    if (lane == 0) out[(I * ntn + Jt) * words + w] = bits;
  }
}

}  // namespace

// The scale-group words of every data tile of an FP8 product (run by the
// encode, which copies the scales; the product only reads them).
cudaError_t launch_f8_groups(const float* sA, const float* sB, int64_t m, int64_t n, int64_t k,
                             uint32_t* out, cudaStream_t st) {
  const int64_t words = cdiv(cdiv(k, 128), 32), ntm = cdiv(m, BM), ntn = cdiv(n, BN);
  const int64_t nw = ntm * ntn * words;
  if (nw == 0) return cudaSuccess;
  k_f8_groups<<<dim3((unsigned)cdiv(ntn * words * 32, 256), (unsigned)std::min<int64_t>(ntm, 65535)),
                256, 0, st>>>(
      sA, sB, cdiv(k, 128), cdiv(n, 128), ntm, ntn, cdiv(k, 128), words, out);
  count_launches(1);
  return cudaGetLastError();
}

namespace {

// ---- host side
PFN_cuTensorMapEncodeTiled_v12000 g_encode_tiled = nullptr;
std::once_flag g_encode_once;
int g_num_sms[64] = {};

cudaError_t get_encoder() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
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

// 2-D fp32 store map of a row-major rows x cols output with leading dimension
// ld: box 32 x 32, 128-byte swizzle (the epilogue's staging layout).  TMA
// needs a 16-byte aligned base and a row pitch that is a multiple of 16
// bytes; otherwise (or for an empty output) there is no map and the
// epilogue stores with plain instructions.  Out-of-range parts of a box are
// not written.
bool make_store_map(CUtensorMap* map, const void* ptr, int64_t rows, int64_t cols, int64_t ld) {
  if (!ptr || rows <= 0 || cols <= 0 || (reinterpret_cast<uintptr_t>(ptr) & 15) || (ld * 4) % 16)
    return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
  const cuuint32_t box[2] = {32, 32};
  const cuuint32_t estr[2] = {1, 1};
  return g_encode_tiled(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(ptr), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 3-D bf16 view of a row-major rows x cols matrix as (64 columns, rows, column
// box): element (x, y, z) is at ptr + y ld + 64 z + x.  Only the cols / 64 full
// boxes are inside the view, so no copy reaches past a row or past the
// matrix; the box is 64 x 64 x depth (depth B boxes of one stage), 128-byte
// swizzle.
bool make_map_boxes(CUtensorMap* map, const void* ptr, int64_t rows, int64_t cols, int64_t ld,
                    int depth = 4) {
  int64_t nb = cols / 64;
  if (rows == 0 || nb == 0) {  // never read: a dummy valid map
    rows = 1;
    nb = 1;
  }
  const cuuint64_t dims[3] = {64, (cuuint64_t)rows, (cuuint64_t)nb};
  const cuuint64_t strides[2] = {(cuuint64_t)(ld * 2), 128};
  const cuuint32_t box[3] = {64, 64, (cuuint32_t)depth};
  const cuuint32_t estr[3] = {1, 1, 1};
  return g_encode_tiled(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(ptr), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// e4m3 (byte) map of the native FP8 data tiles: a row-major rows x cols byte
// matrix with leading dimension ld, box box_cols x box_rows, 128-byte swizzle.
bool make_map_u8(CUtensorMap* map, const void* ptr, int64_t rows, int64_t cols, int64_t ld,
                 uint32_t box_cols, uint32_t box_rows) {
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld};
  const cuuint32_t box[2] = {box_cols, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return g_encode_tiled(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(ptr), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Accumulator promotion: the tensor cores accumulate at most this many
// 64-wide k-steps before the epilogue adds the partial into round-to-nearest
// fp32 registers (0: the whole K loop in one accumulator).  The split products
// exist for accuracy, and the tensor cores' fp32 accumulation over long K
// loops would dominate their error: bf16x6 promotes every 8 steps (measured
// relative error 4.8e-7 at k = 4096 and 16384, below cuBLAS SGEMM's; every 4
// steps gives 2.7e-7 at 5 % lower throughput), bf16x3 every 16 (its 2-piece
// split floor, 4.4e-6, dominates anyway).  Plain bf16 and FP8 do not promote
// by default (measured 12-25 % slower at 16384^3 with it).  The environment
// variable ABFT_PROMOTE_KSTEPS overrides the choice for every dtype.
int promote_ksteps(int dtype) {
  const char* env = getenv("ABFT_PROMOTE_KSTEPS");
  if (env && *env) return std::max(0, atoi(env));
  return dtype == ABFT_BF16X6 ? 8 : (dtype == ABFT_BF16X3 ? 16 : 0);
}

// Raster group height of the single-problem tile order: tiles run column by
// column over groups of this many tile rows (2048 rows), so consecutive CTAs
// share the group's A panels and one B panel in L2.  ABFT_GROUP_M overrides
// the default.
int raster_group_rows(int bm) {
  const char* env = getenv("ABFT_GROUP_M");
  if (env && *env) return std::max(1, atoi(env));
  return 2048 / bm;
}

// Tall (256-row) tiles for products without promotion whose K loop is long
// enough (at least 32 k-steps) that the tile's epilogue, which no longer
// overlaps the next tile's MMAs, is a small share of it.  ABFT_TALL_TILES=0
// or 1 forces the choice.
bool use_tall(int64_t m, int64_t nkt, int kpg) {
  if (kpg > 0) return false;
  const char* env = getenv("ABFT_TALL_TILES");
  if (env && *env) return env[0] == '1';
  return m > BM && nkt >= 32;
}

// Pair tiles (256 x 256 on a CTA pair, see Geo).  Measured at 16384^3 against
// the one-CTA schedules: FP8 (native data tiles) no faster (the MMA warp waits
// on stage data 10 % of the time instead of 17 %, but a pair MMA that does not
// wait runs about 5 % slower per SM than a one-CTA MMA); bf16 10 % slower than
// tall tiles and the promoted bf16x3 / bf16x6 12-20 % slower than regular
// tiles: a pair tile takes half as long as a tall one, so the same drift
// between CTAs puts the tiles that share an operand panel twice as far apart
// in K, and the product reads 17.8 GB from DRAM instead of 7.0; the promoted
// products also wait twice as long for a free accumulator (both CTAs'
// epilogues must release it).  FP8 with pair tiles: 4.097 ms per step against
// 4.099 with regular tiles (the checksum-free product 3.12 against 3.04 ms).  So
// no product uses them unless ABFT_PAIR_TILES=1 asks for them (0 or unset:
// tall or regular tiles).
bool use_pair(int64_t m, bool f8) {
  const char* env = getenv("ABFT_PAIR_TILES");
  (void)m;
  (void)f8;
  return env && env[0] == '1';
}

// Stride of the checksum tiles in the FP8 tile order.  Measured at FP8 16384^3:
// all checksum tiles first (S = 1) 3.18 ms per ABFT product, S = 2 / 3 / 5
// 3.28-3.38 ms, spread over the first 65 % of the schedule 3.35 ms (their
// bf16-plane panels then evict the data tiles' panels from L2).  So S = 1;
// ABFT_FP8_CS_STRIDE sets another stride, and ABFT_FP8_CS_STRIDE=spread the
// spread order (coprime with the grid, every CTA at most ceil(checksum
// tiles / grid) of them).
int64_t cs_stride(int64_t ncs, int64_t total, int grid) {
  const char* env = getenv("ABFT_FP8_CS_STRIDE");
  if (!(env && *env)) return 1;
  if (env[0] != 's') return std::max<int64_t>(1, atoll(env));
  if (ncs <= 0) return 1;
  int64_t S = std::max<int64_t>(1, (total * 65 / 100) / ncs);
  auto gcd = [](int64_t a, int64_t b) {
    while (b) {
      const int64_t r = a % b;
      a = b;
      b = r;
    }
    return a;
  };
  while (S > 1 && gcd(S, grid) != 1) --S;
  return S;
}

// CTA pairs (clusters of two) of a pair-tile kernel that fit on the GPU at
// once: the persistent grid's size.  Clusters are placed within a GPC, so this
// can be less than half the SM count.
int g_pair_clusters[64] = {};
int num_sms();
int pair_clusters(const void* kernel, size_t smem) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && g_pair_clusters[dev]) return g_pair_clusters[dev];
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(2 * (num_sms() / 2), 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kernel, &cfg) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    n = num_sms() / 2;
  }
  if (dev >= 0 && dev < 64) g_pair_clusters[dev] = n;
  return n;
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

// Timeout word of checksum-free products run without a workspace.
__device__ int g_tc_timeout_fallback = 0;

cudaError_t tc_timeout_fallback(int** dev_ptr) {
  return cudaGetSymbolAddress(reinterpret_cast<void**>(dev_ptr), g_tc_timeout_fallback);
}

cudaError_t launch_gemm_bf16(const Plan& P, const TcOperands& op, float* C, void* ws,
                             bool checksums, int* status, cudaStream_t st) {
  cudaError_t e = get_encoder();
  if (e != cudaSuccess) return e;
  const abft_desc& d = P.d;
  const char* w = static_cast<const char*>(ws);
  const int64_t R16 = checksums ? P.L.acs_rows : 0, C16 = checksums ? P.L.bcs_cols : 0;
  TcMaps M;
  // pair tiles: each CTA of a pair copies half of a full tile's B boxes
  const bool pair = use_pair(d.m, op.a8 != nullptr);
  const int bdepth = pair ? 2 : 4;
  for (int pl = 0; pl < kPlanes; ++pl) {
    const int cpl = pl < P.L.planes ? pl : 0;  // checksum planes beyond the dtype's repeat plane 0
    const void* acs = checksums ? w + P.L.acs + cpl * P.L.acs_plane : op.a[0];
    const void* bcs = checksums ? w + P.L.bcs + cpl * P.L.bcs_plane : op.b[0];
    const int64_t acs_ld = checksums ? P.L.acs_ld : op.lda;
    const int64_t bcs_ld = checksums ? P.L.bcs_ld : op.ldb;
    if (!make_map(&M.a[pl], op.a[pl], d.m, d.k, op.lda, 64, BM / 2) ||
        !make_map(&M.acs[pl], acs, R16, d.k, acs_ld, 64, BM / 2) ||
        !make_map(&M.b[pl], op.b[pl], d.k, d.n, op.ldb, 64, BK) ||
        !make_map(&M.bcs[pl], bcs, d.k, C16, bcs_ld, 64, BK) ||
        !make_map(&M.a128[pl], op.a[pl], d.m, d.k, op.lda, 64, BM) ||
        !make_map(&M.acs128[pl], acs, R16, d.k, acs_ld, 64, BM) ||
        !make_map_boxes(&M.b4[pl], op.b[pl], d.k, d.n, op.ldb, bdepth) ||
        !make_map_boxes(&M.bcs4[pl], bcs, d.k, C16, bcs_ld, bdepth))
      return cudaErrorInvalidValue;
  }
  TcArgs g{};
  g.m = d.m; g.n = d.n; g.k = d.k; g.R16 = R16; g.C16 = C16;
  g.st_ok = make_store_map(&M.cst, C, d.m, d.n, d.ldc) ? 1 : 0;
  if (checksums) {
    g.st_ok |= make_store_map(&M.est, w + P.L.E16, R16, d.n, d.n) ? 2 : 0;
    g.st_ok |= make_store_map(&M.fst, w + P.L.F16, d.m, C16, C16) ? 4 : 0;
  }
  g.nseg = op.nseg;
  g.seg_a = op.seg_a;
  g.seg_b = op.seg_b;
  g.kpg = promote_ksteps(d.dtype);
  if (op.a8) {  // native FP8 data tiles on the e4m3 codes (promoted every k-step)
    if (!make_map_u8(&M.a[kF8Slot], op.a8, d.m, d.k, op.lda8, 128, BM / 2) ||
        !make_map_u8(&M.a128[kF8Slot], op.a8, d.m, d.k, op.lda8, 128, BM) ||
        !make_map_u8(&M.b[kF8Slot], op.b8, d.n, d.k, op.ldb8, 128, 64) ||
        !make_map_u8(&M.b4[kF8Slot], op.b8, d.n, d.k, op.ldb8, 128, pair ? BN / 2 : BN))
      return cudaErrorInvalidValue;
    g.f8 = 1;
    g.sA = op.sA;
    g.sB = op.sB;
    g.nsa = cdiv(d.k, 128);
    g.nsb = cdiv(d.n, 128);
    g.kpg = 0;  // the checksum tiles (bf16 planes) run one group
    g.f8grp = op.f8grp;
    g.f8words = cdiv(cdiv(d.k, 128), 32);
  }
  const bool tall = !pair && !g.f8 && use_tall(d.m, cdiv(d.k, BK) * op.nseg, g.kpg);
  const int bm = (tall || pair) ? 256 : BM;
  g.ntm = (int)cdiv(d.m, bm);
  g.ntn = (int)cdiv(d.n, BN);
  g.ntr = checksums ? (int)cdiv(R16, bm) : 0;
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
  g.g = P.g > 0 ? P.g : 128;
  g.ngrp = P.ngrp;
  if (checksums && P.fused) {
    g.obs_col = reinterpret_cast<float*>(const_cast<char*>(w) + P.L.obs_col);
    g.obs_row = reinterpret_cast<float*>(const_cast<char*>(w) + P.L.obs_row);
  }
  if (checksums) {
    g.inj_hdr = reinterpret_cast<const int32_t*>(w + P.L.inject);
    g.inj = reinterpret_cast<const InjectEntry*>(w + P.L.inject + 16);
  }
  g.status = status;
  // Test hook for the bounded waits: ABFT_TEST_STALL_PRODUCER=1 makes the
  // producer skip the first tile, so its MMA wait runs out (after 0.2 s) and
  // the call reports ABFT_ERR_TIMEOUT.  Off unless the variable is set.
  const char* stall = getenv("ABFT_TEST_STALL_PRODUCER");
  g.stall_test = stall && stall[0] == '1';
  g.group_m = raster_group_rows(bm);
  g.wait_ns = g.stall_test ? 200000000ull : tc::kWaitLimitNs;
  const auto kernel =
      pair ? (g.f8 ? k_gemm_bf16<true, false, true, true>
                   : g.kpg > 0 ? k_gemm_bf16<true, false, false, true>
                               : k_gemm_bf16<false, false, false, true>)
           : (g.f8 ? k_gemm_bf16<true, false, true, false>
                   : g.kpg > 0 ? k_gemm_bf16<true, false, false, false>
                               : (tall ? k_gemm_bf16<false, true, false, false>
                                       : k_gemm_bf16<false, false, false, false>));
  const size_t smem =
      pair ? Geo<false, true>::kSmem : (tall ? Geo<true>::kSmem : Geo<false>::kSmem);
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // tile workers: CTAs, or CTA pairs
  const int workers = (int)std::min<int64_t>(
      g.t_total, pair ? pair_clusters(reinterpret_cast<const void*>(kernel), smem) : num_sms());
  if (workers == 0) return cudaSuccess;
  if (g.f8) g.cs_stride = cs_stride(g.t_total - g.t_data, g.t_total, workers);  // 1 unless set
  e = cudaMemsetAsync(status, 0, sizeof(int), st);  // the status of this product
  if (e != cudaSuccess) return e;
  if (pair) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * workers, 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kernel, M, g);
    if (e != cudaSuccess) return e;
  } else {
    kernel<<<workers, kThreads, smem, st>>>(M, g);
  }
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

cudaError_t make_f32_store_map(CUtensorMap* map, const void* ptr, int64_t rows, int64_t cols,
                               int64_t ld, bool* ok) {
  cudaError_t e = get_encoder();
  if (e != cudaSuccess) return e;
  *ok = make_store_map(map, ptr, rows, cols, ld);
  return cudaSuccess;
}

cudaError_t make_bf16_map_boxes(CUtensorMap* map, const void* ptr, int64_t rows, int64_t cols,
                                int64_t ld, int depth) {
  cudaError_t e = get_encoder();
  if (e != cudaSuccess) return e;
  return make_map_boxes(map, ptr, rows, cols, ld, depth) ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_group_gemm(const GroupDev& G, bool checksums, cudaStream_t st) {
  int* status = G.cnt + kCntTimeout;  // the group's own status word
  const int64_t total = checksums ? G.ntiles_cs : G.ntiles_plain;
  const int grid = (int)std::min<int64_t>(total, num_sms());
  if (grid == 0) return cudaSuccess;
  const cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  k_gemm_grouped<<<grid, kThreads, SMEM_BYTES, st>>>(
      G.probs, G.maps, checksums ? G.tiles_cs : G.tiles_plain, total, checksums ? 1 : 0, status,
      tc::kWaitLimitNs, checksums ? G.inj_hdr : nullptr, G.inj, 0);
  count_launches(1);
  return cudaGetLastError();
}

// One-time kernel attributes (outside any stream capture).
cudaError_t prepare_group_kernels() {
  cudaError_t e = get_encoder();
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_gemm_grouped, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)SMEM_BYTES);
}

}  // namespace abft
