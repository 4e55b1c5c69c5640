// Grouped ABFT products: many independent bf16 problems C_p = A_p B_p (each
// with the encoded operands of Eq. (1)) processed by one persistent product
// launch, one encode pass and one verify pass for the whole group.
//
// Host side: validation, the workspace layout (every per-problem region
// carved from the caller's workspace), the device tables (problem records,
// tensor maps, product tile lists, CTA offsets of the grouped kernels), the
// schedule tuning (tile width, problem order) with its measurement-driven
// autotuner and optional cache file, and CUDA-graph capture of the
// product + verify step.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "internal.cuh"

namespace abft {
namespace {

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Per-problem sizes that do not depend on the schedule tuning.
struct ProbShape {
  int64_t nvr, nvc, R16, C16, acs_ld, bcs_ld, nhc, nbc;
  // region offsets inside the workspace
  size_t acs, bcs, E16, F16, obs_col, obs_row, nArow, nAblk, nBcol, nBblk, rowpart, colpart,
      partA, partB, nArow32, nBcol32, tauA, tauB;
  int64_t units[kGkCount];  // CTAs of each grouped kernel
};

}  // namespace
}  // namespace abft

using namespace abft;

struct abft_group_s {
  std::vector<abft_problem> pr;
  std::vector<ProbShape> sh;
  int32_t dtype = ABFT_BF16;
  double s = 4.0;
  abft_group_tuning tune{4, 1};
  // workspace layout
  size_t off_cnt = 0, off_colf = 0, off_rowf = 0, off_cand = 0, off_report = 0, off_inject = 0,
         off_probs = 0, off_maps = 0, off_tiles_cs = 0, off_tiles_plain = 0, off_tab = 0,
         total = 0;
  int64_t ctas[kGkCount] = {};
  int64_t cap_tiles_cs = 0, cap_tiles_plain = 0;
  // bound state
  char* ws = nullptr;
  GroupDev dev{};
  cudaGraphExec_t graph = nullptr;
  int graph_kernels = 0;
};

namespace abft {
namespace {

// Checksum rows of a problem as swapped tiles (kGrpSwapTile): when its data
// rows fill whole 128-row tiles, appended checksum halves would need a tile row
// of their own; a swapped tile's MMA N is the R16 checksum rows (<= 128).
// ABFT_GRP_SWAP=0 keeps the appended halves (for comparison).
bool swap_rows(const abft_problem& p, const ProbShape& s) {
  static const bool on = [] {
    const char* env = getenv("ABFT_GRP_SWAP");
    return !(env && env[0] == '0');
  }();
  return on && cdiv(p.m, 64) % 2 == 0 && s.R16 <= 128;
}

int64_t tiles_of(const abft_problem& p, const ProbShape& s, int bpt, bool cs) {
  const int64_t nhd = cdiv(p.m, 64), nbd = cdiv(p.n, 64);
  const bool sw = cs && swap_rows(p, s);
  const int64_t nh = nhd + (cs && !sw ? s.nhc : 0), nb = nbd + (cs ? s.nbc : 0);
  return cdiv(nh, 2) * cdiv(nb, bpt) + (sw ? cdiv(p.n, 256) : 0);
}

// Problem order of the tile list: as given, or by decreasing inner dimension
// then decreasing tile count (longest tiles first balances the persistent
// round-robin assignment).
std::vector<int> problem_order(const abft_group_s& G, int order) {
  std::vector<int> idx(G.pr.size());
  for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
  if (order == 1)
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
      const abft_problem &x = G.pr[a], &y = G.pr[b];
      if (x.k != y.k) return x.k > y.k;
      return x.m * x.n > y.m * y.n;
    });
  return idx;
}

// Fills the device tables for the current tuning and uploads them (the
// stream is synchronised before the host buffers go away).
abft_status upload_tables(abft_group_s& G, cudaStream_t st) {
  const int count = (int)G.pr.size();
  const int bpt = G.tune.boxes_per_tile;
  char* ws = G.ws;
  std::vector<GProb> probs(count);
  std::vector<GMaps> maps(count);
  std::vector<int2> tab;
  int64_t ntab = 0;
  for (int kk = 0; kk < kGkCount; ++kk) ntab += G.ctas[kk];
  tab.reserve((size_t)ntab);
  for (int kk = 0; kk < kGkCount; ++kk)
    for (int p = 0; p < count; ++p)
      for (int64_t u = 0; u < G.sh[p].units[kk]; ++u) tab.push_back(make_int2(p, (int)u));
  for (int p = 0; p < count; ++p) {
    const abft_problem& q = G.pr[p];
    const ProbShape& s = G.sh[p];
    GProb& P = probs[p];
    memset(&P, 0, sizeof P);
    P.m = q.m; P.n = q.n; P.k = q.k;
    P.lda = q.lda; P.ldb = q.ldb; P.ldc = q.ldc;
    P.A = q.A; P.B = q.B; P.C = static_cast<float*>(q.C);
    P.acs = ws + s.acs; P.bcs = ws + s.bcs;
    P.acs_ld = s.acs_ld; P.bcs_ld = s.bcs_ld; P.R16 = s.R16; P.C16 = s.C16;
    P.E16 = reinterpret_cast<float*>(ws + s.E16);
    P.F16 = reinterpret_cast<float*>(ws + s.F16);
    P.obs_col = reinterpret_cast<float*>(ws + s.obs_col);
    P.obs_row = reinterpret_cast<float*>(ws + s.obs_row);
    P.nArow = reinterpret_cast<double*>(ws + s.nArow);
    P.nAblk = reinterpret_cast<double*>(ws + s.nAblk);
    P.nBcol = reinterpret_cast<double*>(ws + s.nBcol);
    P.nBblk = reinterpret_cast<double*>(ws + s.nBblk);
    P.nArow32 = reinterpret_cast<float*>(ws + s.nArow32);
    P.nBcol32 = reinterpret_cast<float*>(ws + s.nBcol32);
    P.tauA = reinterpret_cast<float*>(ws + s.tauA);
    P.tauB = reinterpret_cast<float*>(ws + s.tauB);
    P.rowpart = reinterpret_cast<float*>(ws + s.rowpart);
    P.colpart = reinterpret_cast<float*>(ws + s.colpart);
    P.partA = reinterpret_cast<double*>(ws + s.partA);
    P.partB = reinterpret_cast<double*>(ws + s.partB);
    P.nvr = s.nvr; P.nvc = s.nvc;
    P.bpt = bpt;
    P.g = 128;  // row-sum groups: one per 128 columns (one epilogue warp's column half)
    P.ngrp = cdiv(q.n, P.g);
    P.nhc = (int32_t)s.nhc; P.nbc = (int32_t)s.nbc;
    P.swap_rows = swap_rows(q, s) ? 1 : 0;
    threshold_factors(G.dtype, q.k, kGrpVbR, kGrpVbC, &P.f1c, &P.f1r, &P.f2);
    cudaError_t e;
    GMaps& Mp = maps[p];
    if ((e = make_bf16_map(&Mp.a, q.A, q.m, q.k, q.lda, 64, 64)) != cudaSuccess ||
        (e = make_bf16_map(&Mp.acs, P.acs, s.R16, q.k, s.acs_ld, 64, 64)) != cudaSuccess ||
        (e = make_bf16_map(&Mp.b, q.B, q.k, q.n, q.ldb, 64, 64)) != cudaSuccess ||
        (e = make_bf16_map(&Mp.bcs, P.bcs, q.k, s.C16, s.bcs_ld, 64, 64)) != cudaSuccess ||
        (e = make_bf16_map(&Mp.a128, q.A, q.m, q.k, q.lda, 64, 128)) != cudaSuccess ||
        (e = make_bf16_map(&Mp.acs128, P.acs, s.R16, q.k, s.acs_ld, 64, 128)) != cudaSuccess ||
        (e = make_bf16_map_boxes(&Mp.bw[0], q.B, q.k, q.n, q.ldb, 2)) != cudaSuccess ||
        (e = make_bf16_map_boxes(&Mp.bw[1], q.B, q.k, q.n, q.ldb, 3)) != cudaSuccess ||
        (e = make_bf16_map_boxes(&Mp.bw[2], q.B, q.k, q.n, q.ldb, 4)) != cudaSuccess ||
        (e = make_bf16_map_boxes(&Mp.bcs4, P.bcs, q.k, s.C16, s.bcs_ld, 4)) != cudaSuccess)
      return fail(ABFT_ERR_INVALID, "problem %d: tensor map rejected (%s)", p,
                  cudaGetErrorString(e));
    // TMA store maps of the outputs (an unaligned C is stored without one)
    bool okc = false, oke = false, okf = false;
    if ((e = make_f32_store_map(&Mp.cst, q.C, q.m, q.n, q.ldc, &okc)) != cudaSuccess ||
        (e = make_f32_store_map(&Mp.est, P.E16, s.R16, q.n, q.n, &oke)) != cudaSuccess ||
        (e = make_f32_store_map(&Mp.fst, P.F16, q.m, s.C16, s.C16, &okf)) != cudaSuccess)
      return fail(ABFT_ERR_INVALID, "problem %d: store map rejected (%s)", p,
                  cudaGetErrorString(e));
    P.st_ok = (okc ? 1 : 0) | (oke ? 2 : 0) | (okf ? 4 : 0);
  }
  // product tile lists
  std::vector<int4> tcs, tpl;
  tcs.reserve((size_t)G.cap_tiles_cs);
  tpl.reserve((size_t)G.cap_tiles_plain);
  for (int p : problem_order(G, G.tune.order)) {
    const abft_problem& q = G.pr[p];
    const ProbShape& s = G.sh[p];
    for (int cs = 0; cs < 2; ++cs) {
      const bool sw = cs && swap_rows(q, s);
      const int64_t nh = cdiv(q.m, 64) + (cs && !sw ? s.nhc : 0),
                    nb = cdiv(q.n, 64) + (cs ? s.nbc : 0);
      const int64_t ntr = cdiv(nh, 2), ntc = cdiv(nb, bpt);
      std::vector<int4>& v = cs ? tcs : tpl;
      const int64_t nbd = cdiv(q.n, 64);
      for (int64_t i = 0; i < ntr; ++i)
        for (int64_t j = 0; j < ntc; ++j) {
          // a tile of one checksum box and no data columns takes two k-steps
          // per stage (kGrpF2Tile)
          const int64_t b0 = bpt * j;
          const bool f2 = cs && b0 >= nbd && std::min<int64_t>(bpt, nb - b0) == 1;
          v.push_back(make_int4(p, (int)i, (int)j, f2 ? kGrpF2Tile : 0));
        }
      // the swapped checksum-row tiles follow the problem's data tiles (its B
      // panels are then still in L2)
      if (sw)
        for (int64_t j = 0; j < cdiv(q.n, 256); ++j)
          v.push_back(make_int4(p, 0, (int)j, kGrpSwapTile));
    }
  }
  if ((int64_t)tcs.size() > G.cap_tiles_cs || (int64_t)tpl.size() > G.cap_tiles_plain)
    return fail(ABFT_ERR_INVALID, "tile list larger than its workspace region");
  cudaError_t e = cudaMemcpyAsync(ws + G.off_probs, probs.data(), sizeof(GProb) * count,
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ws + G.off_maps, maps.data(), sizeof(GMaps) * count,
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !tcs.empty())
    e = cudaMemcpyAsync(ws + G.off_tiles_cs, tcs.data(), sizeof(int4) * tcs.size(),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !tpl.empty())
    e = cudaMemcpyAsync(ws + G.off_tiles_plain, tpl.data(), sizeof(int4) * tpl.size(),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !tab.empty())
    e = cudaMemcpyAsync(ws + G.off_tab, tab.data(), sizeof(int2) * tab.size(),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "abft_group tables");
  GroupDev& D = G.dev;
  D.probs = reinterpret_cast<const GProb*>(ws + G.off_probs);
  D.maps = reinterpret_cast<const GMaps*>(ws + G.off_maps);
  D.count = count;
  D.tiles_cs = reinterpret_cast<const int4*>(ws + G.off_tiles_cs);
  D.ntiles_cs = (int64_t)tcs.size();
  D.tiles_plain = reinterpret_cast<const int4*>(ws + G.off_tiles_plain);
  D.ntiles_plain = (int64_t)tpl.size();
  size_t t0 = 0;
  for (int kk = 0; kk < kGkCount; ++kk) {
    D.tab[kk] = reinterpret_cast<const int2*>(ws + G.off_tab) + t0;
    D.nctas[kk] = G.ctas[kk];
    t0 += (size_t)G.ctas[kk];
  }
  D.s = G.s;
  D.cnt = reinterpret_cast<int32_t*>(ws + G.off_cnt);
  D.colf = reinterpret_cast<FlagEntry*>(ws + G.off_colf);
  D.rowf = reinterpret_cast<FlagEntry*>(ws + G.off_rowf);
  D.cand = reinterpret_cast<CandEntry*>(ws + G.off_cand);
  D.report = reinterpret_cast<abft_fault*>(ws + G.off_report);
  D.inj_hdr = reinterpret_cast<int32_t*>(ws + G.off_inject);
  D.inj = reinterpret_cast<InjectEntry*>(ws + G.off_inject + 16);
  return ABFT_OK;
}

abft_status check_bound(const abft_group_s* G) {
  if (!G) return fail(ABFT_ERR_INVALID, "group is NULL");
  if (!G->ws) return fail(ABFT_ERR_INVALID, "group has no workspace (abft_group_bind)");
  return ABFT_OK;
}

void drop_graph(abft_group_s* G) {
  if (G->graph) cudaGraphExecDestroy(G->graph);
  G->graph = nullptr;
  G->graph_kernels = 0;
}

// Signature of a group for the tuning cache: FNV-1a over the shapes.
uint64_t signature(const abft_group_s& G) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](int64_t v) {
    for (int b = 0; b < 8; ++b) {
      h ^= (uint64_t)((v >> (8 * b)) & 0xff);
      h *= 1099511628211ull;
    }
  };
  mix((int64_t)G.pr.size());
  mix(G.dtype);
  for (const abft_problem& p : G.pr) {
    mix(p.m);
    mix(p.n);
    mix(p.k);
  }
  return h;
}

bool cache_lookup(uint64_t sig, abft_group_tuning* t) {
  const char* path = getenv("ABFT_TUNE_CACHE");
  if (!path || !*path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  unsigned long long s = 0;
  int bpt = 0, order = 0;
  double ms = 0;
  bool found = false;
  while (fscanf(f, "%llx %d %d %lf", &s, &bpt, &order, &ms) == 4)
    if (s == sig && (bpt == 2 || bpt == 4) && (order == 0 || order == 1)) {
      t->boxes_per_tile = bpt;
      t->order = order;
      found = true;
    }
  fclose(f);
  return found;
}

void cache_store(uint64_t sig, const abft_group_tuning& t, double ms) {
  const char* path = getenv("ABFT_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%016llx %d %d %.6f\n", (unsigned long long)sig, t.boxes_per_tile, t.order, ms);
  fclose(f);
}

}  // namespace
}  // namespace abft

extern "C" {

abft_status abft_group_create(const abft_problem* problems, int32_t count, int32_t dtype,
                              double tau_safety, abft_group* out) {
  if (!out) return fail(ABFT_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (count < 0 || (count > 0 && !problems)) return fail(ABFT_ERR_INVALID, "bad problem list");
  if (count >= (1 << 23)) return fail(ABFT_ERR_INVALID, "at most 2^23 - 1 problems");
  if (dtype != ABFT_BF16) return fail(ABFT_ERR_UNSUPPORTED, "grouped products take ABFT_BF16");
  if (!(tau_safety >= 0.0) || !isfinite(tau_safety))
    return fail(ABFT_ERR_INVALID, "tau_safety must be finite and >= 0");
  for (int p = 0; p < count; ++p) {
    const abft_problem& q = problems[p];
    if (q.m < 1 || q.n < 1 || q.k < 1 || q.m > (1 << 20) || q.n > (1 << 20) || q.k > (1 << 24))
      return fail(ABFT_ERR_INVALID, "problem %d: sizes must be m, n in [1, 2^20], k in [1, 2^24]",
                  p);
    if (q.lda < q.k || q.ldb < q.n || q.ldc < q.n || q.lda % 8 || q.ldb % 8)
      return fail(ABFT_ERR_INVALID,
                  "problem %d: need lda >= k, ldb >= n, ldc >= n, lda and ldb multiples of 8", p);
    if (!q.A || !q.B || !q.C) return fail(ABFT_ERR_INVALID, "problem %d: NULL pointer", p);
    if ((reinterpret_cast<uintptr_t>(q.A) | reinterpret_cast<uintptr_t>(q.B)) & 15)
      return fail(ABFT_ERR_INVALID, "problem %d: A and B must be 16-byte aligned", p);
  }
  abft_group_s* G = new abft_group_s;
  G->pr.assign(problems, problems + count);
  G->dtype = dtype;
  G->s = tau_safety > 0 ? tau_safety : 4.0;
  G->sh.resize(count);
  size_t off = 0;
  auto region = [&](size_t bytes) {
    const size_t o = off;
    off = al256(off + bytes);
    return o;
  };
  G->off_cnt = region(256);
  G->off_colf = region(sizeof(FlagEntry) * kCapFlags);
  G->off_rowf = region(sizeof(FlagEntry) * kCapFlags);
  G->off_cand = region(sizeof(CandEntry) * kCapCands);
  G->off_report = region(sizeof(abft_fault) * kCapReport);
  G->off_inject = region(16 + sizeof(InjectEntry) * kMaxInject);
  G->off_probs = region(sizeof(GProb) * count);
  G->off_maps = region(sizeof(GMaps) * count);
  for (int p = 0; p < count; ++p) {
    const abft_problem& q = problems[p];
    ProbShape& s = G->sh[p];
    s.nvr = cdiv(q.m, kGrpVbR);
    s.nvc = cdiv(q.n, kGrpVbC);
    s.R16 = 4 * s.nvr;
    s.C16 = 4 * s.nvc;
    s.acs_ld = (q.k + 7) / 8 * 8;
    s.bcs_ld = (s.C16 + 7) / 8 * 8;
    s.nhc = cdiv(s.R16, 64);
    s.nbc = cdiv(s.C16, 64);
    const int64_t units[kGkCount] = {
        s.nvr * cdiv(s.acs_ld, 256),       // kGkEncA: verify block x 256 columns
        cdiv(q.n, 256) * cdiv(q.k, 128),   // kGkEncB: 256 columns x 128 rows
        cdiv(q.m, 256) + cdiv(q.n, 256),   // kGkLines: 256 rows, then 256 columns
        s.nvr * cdiv(q.n, 256),            // kGkColCheck: verify block x 256 columns
        cdiv(q.m * s.nvc, 256 * kGrpRowLines)};  // kGkRowCheck: 256 threads of kGrpRowLines
    for (int kk = 0; kk < kGkCount; ++kk) {
      s.units[kk] = units[kk];
      G->ctas[kk] += units[kk];
    }
    G->cap_tiles_cs += tiles_of(q, s, 2, true);     // the narrower tile gives the longer list
    G->cap_tiles_plain += tiles_of(q, s, 2, false);
  }
  G->off_tiles_cs = region(sizeof(int4) * G->cap_tiles_cs);
  G->off_tiles_plain = region(sizeof(int4) * G->cap_tiles_plain);
  int64_t ntab = 0;
  for (int kk = 0; kk < kGkCount; ++kk) ntab += G->ctas[kk];
  if (ntab >= (1ll << 31)) {
    delete G;
    return fail(ABFT_ERR_INVALID, "group too large for one launch per kernel");
  }
  G->off_tab = region(sizeof(int2) * ntab);
  for (int p = 0; p < count; ++p) {
    const abft_problem& q = problems[p];
    ProbShape& s = G->sh[p];
    s.acs = region((size_t)s.R16 * s.acs_ld * 2);
    s.bcs = region((size_t)q.k * s.bcs_ld * 2);
    s.E16 = region((size_t)s.R16 * q.n * 4);
    s.F16 = region((size_t)q.m * s.C16 * 4);
    s.obs_col = region((size_t)cdiv(q.m, 32) * 2 * q.n * 4);  // per 32-row block
    s.obs_row = region((size_t)q.m * cdiv(q.n, 128) * 2 * 4);  // groups of >= 128 columns
    s.nArow = region((size_t)q.m * 8);
    s.nAblk = region((size_t)4 * s.nvr * 8);
    s.nBcol = region((size_t)q.n * 8);
    s.nBblk = region((size_t)4 * s.nvc * 8);
    s.rowpart = region((size_t)q.m * cdiv(q.k, 256) * 4);
    s.colpart = region((size_t)cdiv(q.k, 128) * q.n * 4);
    s.partA = region((size_t)2 * s.nvr * cdiv(q.k, 256) * 8);
    s.partB = region((size_t)2 * s.nvc * cdiv(q.k, 128) * 8);
    s.nArow32 = region((size_t)q.m * 4);
    s.nBcol32 = region((size_t)q.n * 4);
    s.tauA = region((size_t)2 * s.nvr * 4);
    s.tauB = region((size_t)2 * s.nvc * 4);
  }
  G->total = off;
  *out = G;
  return ABFT_OK;
}

size_t abft_group_workspace_bytes(abft_group g) { return g ? g->total : 0; }

abft_status abft_group_problem_layout(abft_group g, int32_t p, abft_group_layout* out) {
  if (!g || !out) return fail(ABFT_ERR_INVALID, "NULL argument");
  if (p < 0 || p >= (int32_t)g->pr.size()) return fail(ABFT_ERR_INVALID, "no problem %d", p);
  const ProbShape& s = g->sh[p];
  *out = abft_group_layout{s.acs,   s.bcs,   s.E16,   s.F16, s.obs_col, s.obs_row,
                           s.nArow, s.nAblk, s.nBcol, s.nBblk, s.nvr,   s.nvc,
                           s.R16,   s.C16,   s.acs_ld, s.bcs_ld};
  return ABFT_OK;
}

abft_status abft_group_bind(abft_group g, void* ws, size_t ws_bytes, void* stream) {
  if (!g) return fail(ABFT_ERR_INVALID, "group is NULL");
  if (!ws || ws_bytes < g->total)
    return fail(ABFT_ERR_INVALID, "workspace of %zu bytes needed", g->total);
  if (reinterpret_cast<uintptr_t>(ws) & 255)
    return fail(ABFT_ERR_INVALID, "workspace must be 256-byte aligned");
  cudaError_t e = prepare_group_kernels();
  if (e != cudaSuccess) return cuda_fail(e, "abft_group_bind");
  drop_graph(g);
  g->ws = static_cast<char*>(ws);
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const abft_status s = upload_tables(*g, st);
  if (s != ABFT_OK) {
    g->ws = nullptr;
    return s;
  }
  // disarmed injection list, zeroed counters
  e = cudaMemsetAsync(g->ws + g->off_inject, 0, 16, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->ws + g->off_cnt, 0, 256, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? ABFT_OK : cuda_fail(e, "abft_group_bind");
}

abft_status abft_group_set_tuning(abft_group g, const abft_group_tuning* t, void* stream) {
  abft_status s = check_bound(g);
  if (s != ABFT_OK) return s;
  if (!t || (t->boxes_per_tile != 2 && t->boxes_per_tile != 4) || (t->order != 0 && t->order != 1))
    return fail(ABFT_ERR_INVALID, "tuning: boxes_per_tile 2 or 4, order 0 or 1");
  drop_graph(g);
  g->tune = *t;
  return upload_tables(*g, static_cast<cudaStream_t>(stream));
}

abft_status abft_group_get_tuning(abft_group g, abft_group_tuning* t) {
  if (!g || !t) return fail(ABFT_ERR_INVALID, "NULL argument");
  *t = g->tune;
  return ABFT_OK;
}

abft_status abft_group_encode(abft_group g, void* stream) {
  abft_status s = check_bound(g);
  if (s != ABFT_OK) return s;
  const cudaError_t e = launch_group_encode(g->dev, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? ABFT_OK : cuda_fail(e, "abft_group_encode");
}

abft_status abft_group_gemm(abft_group g, int32_t checksums, void* stream) {
  abft_status s = check_bound(g);
  if (s != ABFT_OK) return s;
  const cudaError_t e = launch_group_gemm(g->dev, checksums != 0, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? ABFT_OK : cuda_fail(e, "abft_group_gemm");
}

abft_status abft_group_verify_enqueue(abft_group g, void* stream) {
  abft_status s = check_bound(g);
  if (s != ABFT_OK) return s;
  const cudaError_t e = launch_group_verify(g->dev, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? ABFT_OK : cuda_fail(e, "abft_group_verify_enqueue");
}

abft_status abft_group_report(abft_group g, abft_fault* report, int32_t max_reports,
                              int32_t* n_reports, void* stream) {
  abft_status s = check_bound(g);
  if (s != ABFT_OK) return s;
  if (n_reports) *n_reports = 0;
  if (max_reports < 0 || (max_reports > 0 && !report))
    return fail(ABFT_ERR_INVALID, "bad report buffer");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  int32_t cnt[kNumCounters];
  cudaError_t e = cudaMemcpyAsync(cnt, g->dev.cnt, sizeof cnt, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "abft_group_report");
  if (cnt[kCntTimeout])  // the group's status word of its last product
    return fail(ABFT_ERR_TIMEOUT,
                "the group's product gave up waiting (bounded wait); results are incomplete and "
                "were not corrected");
  const int total = cnt[kCntReport];
  const int stored = std::min(total, kCapReport);
  std::vector<abft_fault> rep((size_t)stored);
  if (stored > 0) {
    e = cudaMemcpyAsync(rep.data(), g->dev.report, sizeof(abft_fault) * stored,
                        cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "abft_group_report");
  }
  std::sort(rep.begin(), rep.end(), [](const abft_fault& x, const abft_fault& y) {
    if (x.problem != y.problem) return x.problem < y.problem;
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

abft_status abft_group_verify_correct(abft_group g, abft_fault* report, int32_t max_reports,
                                      int32_t* n_reports, void* stream) {
  abft_status s = abft_group_verify_enqueue(g, stream);
  if (s != ABFT_OK) return s;
  return abft_group_report(g, report, max_reports, n_reports, stream);
}

abft_status abft_group_set_epilogue_faults(abft_group g, const int32_t* problem,
                                           const int64_t* rows, const int64_t* cols,
                                           const int32_t* bits, int32_t count, void* stream) {
  abft_status s = check_bound(g);
  if (s != ABFT_OK) return s;
  if (count < 0 || count > kMaxInject || (count > 0 && (!problem || !rows || !cols || !bits)))
    return fail(ABFT_ERR_INVALID, "bad injection list (at most %d entries)", kMaxInject);
  std::vector<InjectEntry> e((size_t)count);
  for (int t = 0; t < count; ++t) {
    const int p = problem[t];
    if (p < 0 || p >= (int)g->pr.size() || rows[t] < 0 || rows[t] >= g->pr[p].m || cols[t] < 0 ||
        cols[t] >= g->pr[p].n || bits[t] < 0 || bits[t] > 31)
      return fail(ABFT_ERR_INVALID, "injection %d outside its problem's C or the fp32 element", t);
    e[(size_t)t] = InjectEntry{(int32_t)rows[t], (int32_t)cols[t], bits[t], p};
  }
  const cudaError_t ce = launch_set_inject_raw(g->dev.inj_hdr, e.data(), count,
                                               static_cast<cudaStream_t>(stream));
  return ce == cudaSuccess ? ABFT_OK : cuda_fail(ce, "abft_group_set_epilogue_faults");
}

abft_status abft_group_capture(abft_group g, int32_t checksums, void* stream) {
  abft_status s = check_bound(g);
  if (s != ABFT_OK) return s;
  drop_graph(g);
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!st) return fail(ABFT_ERR_INVALID, "graph capture needs a non-default stream");
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e, "abft_group_capture");
  const int64_t before = abft_kernel_launches();
  cudaError_t e1 = launch_group_gemm(g->dev, checksums != 0, st);
  if (e1 == cudaSuccess && checksums) e1 = launch_group_verify(g->dev, st);
  e = cudaStreamEndCapture(st, &graph);
  if (e1 != cudaSuccess || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(e1 != cudaSuccess ? e1 : e, "abft_group_capture");
  }
  g->graph_kernels = (int)(abft_kernel_launches() - before);
  count_launches(-(int64_t)g->graph_kernels);  // counted when launched
  e = cudaGraphInstantiate(&g->graph, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    g->graph = nullptr;
    return cuda_fail(e, "abft_group_capture instantiate");
  }
  return ABFT_OK;
}

abft_status abft_group_launch(abft_group g, void* stream) {
  abft_status s = check_bound(g);
  if (s != ABFT_OK) return s;
  if (!g->graph) return fail(ABFT_ERR_INVALID, "no captured graph (abft_group_capture)");
  const cudaError_t e = cudaGraphLaunch(g->graph, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "abft_group_launch");
  count_launches(g->graph_kernels);
  return ABFT_OK;
}

abft_status abft_group_autotune(abft_group g, int32_t reps, abft_group_tuning* chosen,
                                double* best_ms, void* stream) {
  abft_status s = check_bound(g);
  if (s != ABFT_OK) return s;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint64_t sig = signature(*g);
  abft_group_tuning best = g->tune;
  double best_t = -1.0;
  if (cache_lookup(sig, &best)) {
    s = abft_group_set_tuning(g, &best, stream);
    if (s != ABFT_OK) return s;
  } else {
    if (reps < 1) reps = 3;
    const abft_group_tuning cands[4] = {{4, 1}, {4, 0}, {2, 1}, {2, 0}};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
      return fail(ABFT_ERR_CUDA, "abft_group_autotune: events");
    for (const abft_group_tuning& c : cands) {
      s = abft_group_set_tuning(g, &c, stream);
      if (s != ABFT_OK) break;
      cudaError_t e = launch_group_gemm(g->dev, true, st);  // warm-up
      if (e == cudaSuccess) e = cudaEventRecord(e0, st);
      for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_group_gemm(g->dev, true, st);
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        s = cuda_fail(e, "abft_group_autotune");
        break;
      }
      const double t = ms / reps;
      if (best_t < 0 || t < best_t) {
        best_t = t;
        best = c;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != ABFT_OK) return s;
    s = abft_group_set_tuning(g, &best, stream);
    if (s != ABFT_OK) return s;
    cache_store(sig, best, best_t);
  }
  if (chosen) *chosen = best;
  if (best_ms) *best_ms = best_t;
  return ABFT_OK;
}

abft_status abft_group_destroy(abft_group g) {
  if (!g) return ABFT_OK;
  drop_graph(g);
  delete g;
  return ABFT_OK;
}

}  // extern "C"
