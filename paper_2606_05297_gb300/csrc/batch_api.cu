// batch_api.cu -- host side of the batched engine (cvq_batch_*): per-instance
// buffers, the layer and work-item schedule of one ansatz structure, the
// final reduction plan, and the CUDA graph that replays one evaluation.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "cvq_internal.cuh"
#include "k_ham_impl.cuh"
#include "k_tile_impl.cuh"

namespace cvq {
int internal_fail(int code, const char* msg);
const SectorDev* internal_sector(const cvq_sector* s);
int internal_sector_device(const cvq_sector* s);
int internal_pool_host(const cvq_pool* p, const cvq_sector** sec, const TypeDesc** types, int* ntypes,
                       const int** op_type, const int** op_i, const int** op_j, int* K, PoolDev* P, int* ustride,
                       const GateArg** ops_dev, const TileMap** op_tiles);
int internal_screen_plan(const cvq_pool* p, const int* subset, int n_subset, ScreenArg* sa, ScreenMap* sm);
}  // namespace cvq

using namespace cvq;

namespace {

struct PoolView {
  const cvq_sector* sec;
  const TypeDesc* types;
  int ntypes, K, ustride;
  const int *op_type, *op_i, *op_j;
  PoolDev P;
  const GateArg* ops_dev;
  const TileMap* op_tiles;  // host copy of each operator's tiles (NULL: no tiles)
};

int errf(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  return internal_fail(code, buf);
}

int cuda_err(cudaError_t e, const char* what) {
  const int code = cvq_status_from_cuda((int)e);
  return errf(code == CVQ_OK ? CVQ_ECUDA : code, "%s: %s", what, cudaGetErrorString(e));
}

#define BCUDA(call, what)                             \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_err(e_, what); \
  } while (0)

size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

// Shared memory one CTA of the small-instance kernel may use (tables + psi + lambda).
constexpr int kSmallSmem = 160 * 1024;

}  // namespace

struct cvq_batch {
  int n = 0, kind = 0, device = 0, n_max = 0, sms = 0;
  std::vector<PoolView> pv;
  std::vector<SectorDev> S;
  void* state = nullptr;  // psi, lam, U of every instance
  std::vector<BInst> inst;
  BInst* inst_d = nullptr;
  // schedule knobs
  int64_t tile = 32768;   // amplitudes per work item
  int ctas_per_sm = 2;
  // structure
  bool have = false;
  std::vector<int> n_ops, ids;  // host copy (rebuilds on schedule changes)
  std::vector<const double2*> psi0;
  void* plan = nullptr;         // ids, segments, items, reductions, gates, counters, partials
  int* ids_d = nullptr;
  BSeg* segs_d = nullptr;
  BItem* items_d = nullptr;
  BRed* red_d = nullptr;
  int2* gates_d = nullptr;
  int* counters_d = nullptr;
  int* active_d = nullptr;                 // per instance: 1 = evaluated
  std::vector<std::vector<int4>> chunks;   // host copy of every BH pool's chunk schedule
  double* partial_d = nullptr;
  std::vector<int> layer_off, layer_n;
  std::vector<char> layer_adj;
  std::vector<char> layer_tile;  // every item is a tile range (k_batch_tile_layer)
  int n_red = 0, n_gates = 0, n_items = 0, n_theta = 0;
  size_t smem = 0;       // dynamic shared memory of the generic layer kernel
  size_t tile_smem = 0;  // of the tile-only layer kernel (0: no pool has one-slot tile tables)
  size_t gen_smem = 0;   // gate tables without tile items (the small-instance kernel's table region)
  int maxblk = 0;  // most blocks of any block-gate type of the batch's pools
  // every sector fits one CTA's shared memory: one CTA per instance runs the
  // whole evaluation (k_batch_small) instead of one launch per layer
  bool small = false;
  size_t small_smem = 0;
  // graph
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  const double* g_theta = nullptr;
  double *g_E = nullptr, *g_grad = nullptr;
  // batched screen: its own plan and graph (forward layers of the evaluation
  // plan, then the screen layer, the reduction into z and the epilogue)
  std::vector<const cvq_pool*> pools;
  void* splan = nullptr;
  cudaGraphExec_t sexec = nullptr;
  bool s_valid = false;           // the screen plan matches the current ansatz structure and schedule
  std::vector<int> s_key;         // the subsets it was built for
  const double* s_theta = nullptr;
  double* s_grad = nullptr;
  int* s_counters = nullptr;
  BScreen* s_screens = nullptr;
  int4* s_desc = nullptr;
  BItem* s_items = nullptr;
  BRed* s_red = nullptr;
  BScreenOut* s_outs = nullptr;
  double *s_partial = nullptr, *s_z = nullptr;
  int s_nitems = 0, s_nred = 0, s_nouts = 0;
};

namespace {

void drop_graph(cvq_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
}

void drop_screen(cvq_batch* b) {
  if (b->sexec) cudaGraphExecDestroy(b->sexec);
  b->sexec = nullptr;
  if (b->splan) cudaFree(b->splan);
  b->splan = nullptr;
  b->s_valid = false;
}

// The segments of one instance: a block gate alone, or a run of consecutive
// diagonal gates (at most BATCH_RUN, at most MAX_RUN_PAIRS cross-Kerr).
std::vector<BSeg> segments_of(const PoolView& p, int inst, const int* ids, int n) {
  std::vector<BSeg> v;
  int k = 0;
  while (k < n) {
    BSeg s;
    memset(&s, 0, sizeof s);
    s.inst = inst;
    s.k0 = k;
    const TypeDesc& t0 = p.types[p.op_type[ids[k]]];
    if (!t0.diag) {
      s.m = 1;
      v.push_back(s);
      ++k;
      continue;
    }
    s.isdiag = 1;
    while (k + s.m < n && s.m < BATCH_RUN) {
      const int op = ids[k + s.m];
      const TypeDesc& t = p.types[p.op_type[op]];
      if (!t.diag) break;
      if (t.diag == 4) {
        if (s.npair == MAX_RUN_PAIRS) break;
        s.pi[s.npair] = p.op_i[op];
        s.pj[s.npair] = p.op_j[op];
        ++s.npair;
      }
      s.diag[s.m] = t.diag;
      s.gi[s.m] = p.op_i[op];
      s.gj[s.m] = p.op_j[op];
      ++s.m;
    }
    bool on[LMAX] = {};
    for (int q = 0; q < s.m; ++q)
      if (s.diag[q] != 4) on[s.gi[q]] = true;
    for (int r = 0; r < LMAX; ++r)
      if (on[r]) s.act[s.nact++] = r;
    v.push_back(s);
    k += s.m;
  }
  return v;
}

// Work items of one segment (or of a whole-sector pass when seg < 0).
void items_of(const cvq_batch* b, int inst, int seg, const BSeg* sg, int kind, std::vector<BItem>& out, int& slot,
              int slots_per_item) {
  const SectorDev& S = b->S[inst];
  const PoolView& p = b->pv[inst];
  auto push = [&](int64_t a, int64_t e) {
    BItem it;
    it.kind = kind;
    it.inst = inst;
    it.seg = seg;
    it.slot = slot;
    slot += slots_per_item;
    it.a = a;
    it.b = e;
    out.push_back(it);
  };
  if (kind != BI_GATE) {
    for (int64_t x = 0; x < S.dim; x += b->tile) push(x, std::min<int64_t>(S.dim, x + b->tile));
    return;
  }
  // the pool operator of this block gate
  const int op = b->ids[(size_t)b->inst[inst].ids_off + sg->k0];
  const TypeDesc& t = p.types[p.op_type[op]];
  // tiled gate of one slot per thread (the layer kernel's register budget
  // holds no more): ranges of about `tile` table slots
  if (p.op_tiles && p.op_tiles[op].idx && p.op_tiles[op].slots == 1) {
    const TileMap& tm = p.op_tiles[op];
    const int64_t per = std::max<int64_t>(1, b->tile / ((int64_t)TILE_T * tm.slots));
    for (int64_t u = 0; u < tm.ntiles; u += per) {
      push(u, std::min<int64_t>(tm.ntiles, u + per));
      out.back().kind = BI_TILE;
    }
    return;
  }
  if (S.kind == CVQ_BKC) {
    const int nm = t.single ? 1 : 2;
    int64_t items = 1, per_orbit = 1;
    for (int r = 0; r < S.L - nm; ++r) items *= S.D;
    for (int r = 0; r < nm; ++r) per_orbit *= S.D;
    per_orbit = std::max<int64_t>(1, per_orbit / 2);
    const int64_t orbits = std::max<int64_t>(NTHREADS, b->tile / per_orbit);
    for (int64_t u = 0; u < items; u += orbits) push(u, std::min(items, u + orbits));
  } else {
    // consecutive equal-work chunks until the item holds about `tile` amplitudes
    const int4* ch = b->chunks[inst].data() + t.chunk_base;
    int64_t acc = 0, c0 = 0;
    for (int c = 0; c < t.nchunks; ++c) {
      acc += (int64_t)(ch[c].z - ch[c].y) * (ch[c].x + 1);
      if (acc >= b->tile || c + 1 == t.nchunks) {
        push(c0, c + 1);
        c0 = c + 1;
        acc = 0;
      }
    }
  }
}

int build_plan(cvq_batch* b) {
  drop_graph(b);
  drop_screen(b);
  if (b->plan) cudaFree(b->plan);
  b->plan = nullptr;
  const int n = b->n;
  // instance offsets into ids / theta / grad
  int off = 0;
  std::vector<std::vector<BSeg>> segs(n);
  int smax = 0;
  for (int i = 0; i < n; ++i) {
    b->inst[i].ids_off = off;
    b->inst[i].theta_off = off;
    b->inst[i].psi0 = b->psi0[i];
    if (b->n_ops[i] > 0) segs[i] = segments_of(b->pv[i], i, b->ids.data() + off, b->n_ops[i]);
    smax = std::max(smax, (int)segs[i].size());
    off += std::max(b->n_ops[i], 0);
  }
  b->n_theta = off;
  std::vector<BSeg> seg_all;
  std::vector<std::vector<int>> seg_id(n);
  for (int i = 0; i < n; ++i) {
    b->inst[i].seg0 = (int)seg_all.size();
    b->inst[i].nseg = (b->n_ops[i] < 0) ? -1 : (int)segs[i].size();
    for (auto& s : segs[i]) {
      seg_id[i].push_back((int)seg_all.size());
      seg_all.push_back(s);
    }
  }
  // layers: conversion, smax forward, matvec, smax reverse
  std::vector<std::vector<BItem>> layers(2 * smax + 2);
  std::vector<char> adj(2 * smax + 2, 0);
  std::vector<BRed> red;
  int slot = 0, nosl = 0;
  for (int i = 0; i < n; ++i)
    if (b->n_ops[i] >= 0) items_of(b, i, -1, nullptr, BI_TODF, layers[0], nosl, 0);
  for (int l = 0; l < smax; ++l)
    for (int i = 0; i < n; ++i) {
      if (l >= (int)segs[i].size()) continue;
      const BSeg& s = segs[i][l];
      items_of(b, i, seg_id[i][l], &s, s.isdiag ? BI_DIAG : BI_GATE, layers[1 + l], nosl, 0);
    }
  for (int i = 0; i < n; ++i) {
    if (b->n_ops[i] < 0) continue;
    const int s0 = slot;
    const size_t before = layers[smax + 1].size();
    items_of(b, i, -1, nullptr, BI_APPLYH, layers[smax + 1], slot, 1);
    red.push_back({i, i, 1, s0, (int)(layers[smax + 1].size() - before), 1});
  }
  for (int r = 0; r < smax; ++r) {
    const int l = smax + 2 + r;
    adj[l] = 1;
    for (int i = 0; i < n; ++i) {
      const int ns = (int)segs[i].size();
      if (r >= ns) continue;
      const BSeg& s = segs[i][ns - 1 - r];
      const int s0 = slot;
      const size_t before = layers[l].size();
      items_of(b, i, seg_id[i][ns - 1 - r], &s, s.isdiag ? BI_DIAG : BI_GATE, layers[l], slot, s.m);
      const int cnt = (int)(layers[l].size() - before);
      for (int q = 0; q < s.m; ++q) red.push_back({i, b->inst[i].theta_off + s.k0 + q, 0, s0 + q, cnt, s.m});
    }
  }
  std::vector<int2> gates;
  for (int i = 0; i < n; ++i)
    for (auto& s : segs[i])
      if (!s.isdiag) gates.push_back(make_int2(i, s.k0));
  std::vector<BItem> items;
  b->layer_off.clear();
  b->layer_n.clear();
  b->layer_adj.clear();
  b->layer_tile.clear();
  for (size_t l = 0; l < layers.size(); ++l) {
    b->layer_off.push_back((int)items.size());
    b->layer_n.push_back((int)layers[l].size());
    b->layer_adj.push_back(adj[l]);
    bool tile_only = !layers[l].empty();
    for (const BItem& it : layers[l]) tile_only = tile_only && it.kind == BI_TILE;
    b->layer_tile.push_back(tile_only ? 1 : 0);
    items.insert(items.end(), layers[l].begin(), layers[l].end());
  }
  b->n_items = (int)items.size();
  b->n_red = (int)red.size();
  b->n_gates = (int)gates.size();
  // one device allocation for the whole plan
  const size_t s_ids = a256(sizeof(int) * std::max<size_t>(1, b->ids.size()));
  const size_t s_seg = a256(sizeof(BSeg) * std::max<size_t>(1, seg_all.size()));
  const size_t s_it = a256(sizeof(BItem) * std::max<size_t>(1, items.size()));
  const size_t s_red = a256(sizeof(BRed) * std::max<size_t>(1, red.size()));
  const size_t s_g = a256(sizeof(int2) * std::max<size_t>(1, gates.size()));
  const size_t s_c = a256(sizeof(int) * layers.size());
  const size_t s_a = a256(sizeof(int) * n);
  const size_t s_p = a256(sizeof(double) * std::max(1, slot));
  BCUDA(cudaMalloc(&b->plan, s_ids + s_seg + s_it + s_red + s_g + s_c + s_a + s_p), "cudaMalloc of the batch plan");
  char* q = (char*)b->plan;
  b->ids_d = (int*)q;
  q += s_ids;
  b->segs_d = (BSeg*)q;
  q += s_seg;
  b->items_d = (BItem*)q;
  q += s_it;
  b->red_d = (BRed*)q;
  q += s_red;
  b->gates_d = (int2*)q;
  q += s_g;
  b->counters_d = (int*)q;
  q += s_c;
  b->active_d = (int*)q;
  q += s_a;
  b->partial_d = (double*)q;
  if (!b->ids.empty()) BCUDA(cudaMemcpy(b->ids_d, b->ids.data(), sizeof(int) * b->ids.size(), cudaMemcpyHostToDevice), "copy ids");
  if (!seg_all.empty()) BCUDA(cudaMemcpy(b->segs_d, seg_all.data(), sizeof(BSeg) * seg_all.size(), cudaMemcpyHostToDevice), "copy segments");
  if (!items.empty()) BCUDA(cudaMemcpy(b->items_d, items.data(), sizeof(BItem) * items.size(), cudaMemcpyHostToDevice), "copy items");
  if (!red.empty()) BCUDA(cudaMemcpy(b->red_d, red.data(), sizeof(BRed) * red.size(), cudaMemcpyHostToDevice), "copy reductions");
  if (!gates.empty()) BCUDA(cudaMemcpy(b->gates_d, gates.data(), sizeof(int2) * gates.size(), cudaMemcpyHostToDevice), "copy gates");
  BCUDA(cudaMemcpy(b->inst_d, b->inst.data(), sizeof(BInst) * n, cudaMemcpyHostToDevice), "copy instances");
  std::vector<int> act(n);
  for (int i = 0; i < n; ++i) act[i] = b->n_ops[i] >= 0;
  BCUDA(cudaMemcpy(b->active_d, act.data(), sizeof(int) * n, cudaMemcpyHostToDevice), "copy active flags");
  b->have = true;
  return CVQ_OK;
}

int finish_capture(cvq_batch* b, cudaStream_t st, cudaError_t e, const double* theta, double* E, double* grad) {
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(st, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_err(e != cudaSuccess ? e : e2, "capture of the batch evaluation");
  }
  e = cudaGraphInstantiate(&b->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    b->exec = nullptr;
    return cuda_err(e, "graph instantiation");
  }
  b->g_theta = theta;
  b->g_E = E;
  b->g_grad = grad;
  return CVQ_OK;
}

int capture(cvq_batch* b, const double* theta, double* E, double* grad) {
  drop_graph(b);
  cudaStream_t st = b->cap;
  BCUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
  cudaError_t e = cudaSuccess;
  if (b->small) {
    e = launch_batch_build(b->inst_d, b->gates_d, b->n_gates, b->maxblk, b->ids_d, theta, b->active_d, st);
    if (e == cudaSuccess)
      e = launch_batch_small(b->kind, 0, b->n, b->gen_smem, std::max(b->n_max, 1), b->small_smem, b->inst_d, b->segs_d,
                             b->ids_d, theta, b->active_d, E, grad, st);
    return finish_capture(b, st, e, theta, E, grad);
  }
  e = cudaMemsetAsync(b->counters_d, 0, sizeof(int) * b->layer_n.size(), st);
  if (e == cudaSuccess) e = launch_batch_build(b->inst_d, b->gates_d, b->n_gates, b->maxblk, b->ids_d, theta, b->active_d, st);
  // a layer needs no more CTAs than it has items (small instances leave most of the grid idle)
  const int grid_max = b->sms * b->ctas_per_sm;
  for (size_t l = 0; l < b->layer_n.size() && e == cudaSuccess; ++l) {
    if (b->layer_tile[l])
      e = launch_batch_tile_layer(b->layer_adj[l] != 0, std::min(b->sms * 5, b->layer_n[l]), b->tile_smem, b->inst_d,
                                  b->segs_d, b->items_d + b->layer_off[l], b->layer_n[l], b->counters_d + l, b->ids_d,
                                  b->active_d, b->partial_d, st);
    else
      e = launch_batch_layer(b->kind, b->layer_adj[l] != 0, std::min(grid_max, b->layer_n[l]), b->smem, b->inst_d,
                             b->segs_d, b->items_d + b->layer_off[l], b->layer_n[l], b->counters_d + l, b->ids_d,
                             theta, b->active_d, b->partial_d, st);
  }
  if (e == cudaSuccess) e = launch_batch_reduce(b->red_d, b->n_red, b->partial_d, b->active_d, E, grad, st);
  return finish_capture(b, st, e, theta, E, grad);
}

// The plan of the batched screen for the given subsets (subset_off == NULL:
// every instance's whole pool): per instance its distinct shifts and diagonal
// functions, work items of about `tile` amplitudes, the reduction of their
// partials into z rows and one epilogue entry per screened element.
int build_screen_plan(cvq_batch* b, const int* subset_off, const int* subset) {
  drop_screen(b);
  const int n = b->n;
  std::vector<BScreen> scr(n);
  std::vector<int4> desc;
  std::vector<BItem> items;
  std::vector<BRed> red;
  std::vector<BScreenOut> outs;
  std::vector<ScreenArg> sa(1);
  std::vector<ScreenMap> sm(1);
  int slot = 0, zrows = 0;
  for (int i = 0; i < n; ++i) {
    memset(&scr[i], 0, sizeof(BScreen));
    if (b->n_ops[i] < 0) continue;
    const int* sub = subset_off ? subset + subset_off[i] : nullptr;
    const int ns = subset_off ? subset_off[i + 1] - subset_off[i] : 0;
    if (int rc = internal_screen_plan(b->pools[i], sub, ns, sa.data(), sm.data())) return rc;
    const ScreenArg& A = sa[0];
    const ScreenMap& M = sm[0];
    scr[i].sh_off = (int)desc.size();
    scr[i].nsh = A.nsh;
    desc.insert(desc.end(), A.sh, A.sh + A.nsh);
    scr[i].dg_off = (int)desc.size();
    scr[i].ndg = A.ndg;
    desc.insert(desc.end(), A.dg, A.dg + A.ndg);
    const int rows = 2 * A.nsh + A.ndg;
    if (rows > 0) {
      const int s0 = slot;
      int cnt = 0;
      for (int64_t x = 0; x < b->S[i].dim; x += b->tile, ++cnt) {
        BItem it;
        it.kind = BI_APPLYH;  // unused by the screen kernel
        it.inst = i;
        it.seg = -1;
        it.slot = slot;
        it.a = x;
        it.b = std::min<int64_t>(b->S[i].dim, x + b->tile);
        items.push_back(it);
        slot += rows;
      }
      for (int r = 0; r < rows; ++r) red.push_back({i, zrows + r, 1, s0 + r, cnt, rows});
    }
    for (int k = 0; k < M.n; ++k) {
      BScreenOut o;
      memset(&o, 0, sizeof o);
      o.inst = i;
      o.zrow = zrows;
      o.out = (int)outs.size();
      o.isdg = M.e[k].x;
      o.sp = M.e[k].y;
      o.sn = M.e[k].z;
      o.d = 2 * A.nsh + M.e[k].y;  // diagonal sums follow the 2 nsh shift rows
      o.cp = M.cp[k];
      outs.push_back(o);
    }
    zrows += rows;
  }
  const int nl = (int)b->layer_n.size();
  const size_t s_c = a256(sizeof(int) * (nl + 1));
  const size_t s_s = a256(sizeof(BScreen) * n);
  const size_t s_d = a256(sizeof(int4) * std::max<size_t>(1, desc.size()));
  const size_t s_i = a256(sizeof(BItem) * std::max<size_t>(1, items.size()));
  const size_t s_r = a256(sizeof(BRed) * std::max<size_t>(1, red.size()));
  const size_t s_o = a256(sizeof(BScreenOut) * std::max<size_t>(1, outs.size()));
  const size_t s_p = a256(sizeof(double) * std::max(1, slot));
  const size_t s_z = a256(sizeof(double) * std::max(1, zrows));
  BCUDA(cudaMalloc(&b->splan, s_c + s_s + s_d + s_i + s_r + s_o + s_p + s_z), "cudaMalloc of the screen plan");
  char* q = (char*)b->splan;
  b->s_counters = (int*)q;
  q += s_c;
  b->s_screens = (BScreen*)q;
  q += s_s;
  b->s_desc = (int4*)q;
  q += s_d;
  b->s_items = (BItem*)q;
  q += s_i;
  b->s_red = (BRed*)q;
  q += s_r;
  b->s_outs = (BScreenOut*)q;
  q += s_o;
  b->s_partial = (double*)q;
  q += s_p;
  b->s_z = (double*)q;
  BCUDA(cudaMemcpy(b->s_screens, scr.data(), sizeof(BScreen) * n, cudaMemcpyHostToDevice), "copy screens");
  if (!desc.empty()) BCUDA(cudaMemcpy(b->s_desc, desc.data(), sizeof(int4) * desc.size(), cudaMemcpyHostToDevice), "copy shifts");
  if (!items.empty()) BCUDA(cudaMemcpy(b->s_items, items.data(), sizeof(BItem) * items.size(), cudaMemcpyHostToDevice), "copy items");
  if (!red.empty()) BCUDA(cudaMemcpy(b->s_red, red.data(), sizeof(BRed) * red.size(), cudaMemcpyHostToDevice), "copy reductions");
  if (!outs.empty()) BCUDA(cudaMemcpy(b->s_outs, outs.data(), sizeof(BScreenOut) * outs.size(), cudaMemcpyHostToDevice), "copy outputs");
  b->s_nitems = (int)items.size();
  b->s_nred = (int)red.size();
  b->s_nouts = (int)outs.size();
  b->s_valid = true;
  return CVQ_OK;
}

int capture_screen(cvq_batch* b, const double* theta, double* grad) {
  if (b->sexec) cudaGraphExecDestroy(b->sexec);
  b->sexec = nullptr;
  cudaStream_t st = b->cap;
  const int nl = (int)b->layer_n.size();
  const int nfwd = nl / 2 + 1;  // conversion, forward segments, matvec
  BCUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
  cudaError_t e = cudaMemsetAsync(b->s_counters, 0, sizeof(int) * (nl + 1), st);
  if (e == cudaSuccess) e = launch_batch_build(b->inst_d, b->gates_d, b->n_gates, b->maxblk, b->ids_d, theta, b->active_d, st);
  const int grid = b->sms * b->ctas_per_sm;
  if (b->small && e == cudaSuccess)  // forward sweep and H psi of every instance, one CTA each
    e = launch_batch_small(b->kind, 1, b->n, b->gen_smem, std::max(b->n_max, 1), b->small_smem, b->inst_d, b->segs_d,
                           b->ids_d, theta, b->active_d, nullptr, nullptr, st);
  for (int l = 0; l < nfwd && e == cudaSuccess && !b->small; ++l) {
    if (b->layer_tile[l])
      e = launch_batch_tile_layer(false, std::min(b->sms * 5, b->layer_n[l]), b->tile_smem, b->inst_d, b->segs_d,
                                  b->items_d + b->layer_off[l], b->layer_n[l], b->s_counters + l, b->ids_d,
                                  b->active_d, b->partial_d, st);
    else
      e = launch_batch_layer(b->kind, false, std::min(grid, b->layer_n[l]), b->smem, b->inst_d, b->segs_d,
                             b->items_d + b->layer_off[l], b->layer_n[l], b->s_counters + l, b->ids_d, theta,
                             b->active_d, b->partial_d, st);
  }
  if (e == cudaSuccess)
    e = launch_batch_screen(b->kind, std::min(grid, b->s_nitems), b->inst_d, b->s_items, b->s_nitems,
                            b->s_counters + nl, b->active_d,
                            b->s_screens, b->s_desc, b->s_partial, st);
  if (e == cudaSuccess) e = launch_batch_reduce(b->s_red, b->s_nred, b->s_partial, b->active_d, b->s_z, nullptr, st);
  if (e == cudaSuccess) e = launch_batch_screen_out(b->s_outs, b->s_nouts, b->s_z, b->active_d, grad, st);
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(st, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_err(e != cudaSuccess ? e : e2, "capture of the batched screen");
  }
  e = cudaGraphInstantiate(&b->sexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    b->sexec = nullptr;
    return cuda_err(e, "graph instantiation");
  }
  b->s_theta = theta;
  b->s_grad = grad;
  return CVQ_OK;
}

}  // namespace

extern "C" int cvq_batch_screen(cvq_batch* b, const double* theta_dev, const int* subset_off, const int* subset,
                                double* grad_dev, void* stream) {
  if (!b || !grad_dev) return errf(CVQ_EINVAL, "null argument");
  if (!b->have) return errf(CVQ_EINVAL, "cvq_batch_set_ansatz has not been called");
  if (b->n_theta > 0 && !theta_dev) return errf(CVQ_EINVAL, "null theta");
  std::vector<int> key;
  if (subset_off) {
    if (subset_off[0] != 0) return errf(CVQ_EINVAL, "subset_off[0] must be 0");
    for (int i = 0; i < b->n; ++i)
      if (subset_off[i + 1] < subset_off[i]) return errf(CVQ_EINVAL, "subset_off decreases at instance %d", i);
    if (subset_off[b->n] > 0 && !subset) return errf(CVQ_EINVAL, "null subset");
    key.assign(subset_off, subset_off + b->n + 1);
    key.insert(key.end(), subset, subset + subset_off[b->n]);
  } else {
    key.push_back(-1);
  }
  if (!b->s_valid || key != b->s_key) {
    if (int rc = build_screen_plan(b, subset_off, subset)) {
      drop_screen(b);
      return rc;
    }
    b->s_key = key;
  }
  if (!b->sexec || b->s_theta != theta_dev || b->s_grad != grad_dev)
    if (int rc = capture_screen(b, theta_dev, grad_dev)) return rc;
  BCUDA(cudaGraphLaunch(b->sexec, (cudaStream_t)stream), "graph launch");
  return CVQ_OK;
}

extern "C" int cvq_batch_create(const cvq_sector* const* sectors, const cvq_pool* const* pools, int n_inst, int n_max,
                                cvq_batch** out) {
  if (!out || !sectors || !pools) return errf(CVQ_EINVAL, "null argument");
  *out = nullptr;
  if (n_inst < 1 || n_inst > 4096) return errf(CVQ_EINVAL, "n_inst %d outside [1, 4096]", n_inst);
  if (n_max < 0 || n_max > MAX_GATES) return errf(CVQ_EINVAL, "n_max %d outside [0, %d]", n_max, MAX_GATES);
  cvq_batch* b = new (std::nothrow) cvq_batch;
  if (!b) return errf(CVQ_ENOMEM, "host allocation");
  b->n = n_inst;
  b->n_max = n_max;
  b->pools.assign(pools, pools + n_inst);
  b->pv.resize(n_inst);
  b->S.resize(n_inst);
  b->inst.resize(n_inst);
  size_t total = 0;
  std::vector<size_t> offs(n_inst);
  size_t smem = std::max(sizeof(HSmem), (size_t)(LMAX * DMAX + MAX_RUN_PAIRS * DMAX * DMAX) * sizeof(cdf));
  size_t tsmem = 0;  // tile items (generic layer kernel, and the tile-only one)
  for (int i = 0; i < n_inst; ++i) {
    PoolView& p = b->pv[i];
    int rc = internal_pool_host(pools[i], &p.sec, &p.types, &p.ntypes, &p.op_type, &p.op_i, &p.op_j, &p.K, &p.P,
                                &p.ustride, &p.ops_dev, &p.op_tiles);
    if (rc || p.sec != sectors[i]) {
      delete b;
      return rc ? rc : errf(CVQ_EINVAL, "pool %d belongs to another sector", i);
    }
    const SectorDev* S = internal_sector(sectors[i]);
    if (!S) {
      delete b;
      return errf(CVQ_EINVAL, "null sector %d", i);
    }
    if (i == 0) {
      b->kind = S->kind;
      b->device = internal_sector_device(sectors[i]);
    } else if (S->kind != b->kind || internal_sector_device(sectors[i]) != b->device) {
      delete b;
      return errf(CVQ_EINVAL, "instance %d differs in sector kind or device", i);
    }
    b->S[i] = *S;
    for (int t = 0; t < p.ntypes; ++t)
      if (!p.types[t].diag) {
        smem = std::max(smem, gate_smem_bytes(p.types[t], S->kind));
        b->maxblk = std::max(b->maxblk, p.types[t].nblocks);
      }
    for (int k = 0; p.op_tiles && k < p.K; ++k) {
      const TileMap& tm = p.op_tiles[k];
      if (tm.idx && tm.slots == 1)
        tsmem = std::max(tsmem, tile_smem_bytes(p.types[p.op_type[k]], tm.nreg, tm.nsub, true, 1));
    }
    offs[i] = total;
    total += 2 * a256(sizeof(cdf) * (size_t)S->dim) + a256(sizeof(cdf) * (size_t)std::max(n_max, 1) * p.ustride);
  }
  if (std::max(smem, tsmem) > 200 * 1024) {
    delete b;
    return errf(CVQ_EINVAL, "gate tables need %zu bytes of shared memory", std::max(smem, tsmem));
  }
  {
    int64_t dmax = 0;
    for (int i = 0; i < n_inst; ++i) dmax = std::max<int64_t>(dmax, b->S[i].dim);
    // the generic layer kernel also holds the Bose-Hubbard items' walk buffer
    const size_t walk = (b->kind == CVQ_BH) ? batch_walk_offset() + BATCH_WALK_BYTES : 0;
    b->smem = a256(std::max(std::max(smem, tsmem), walk));
    b->tile_smem = tsmem ? a256(tsmem) : 0;
    b->gen_smem = a256(smem);
    // every instance has at most n_max segments (the small-instance kernel runs no tile items)
    const size_t need = batch_small_smem(b->gen_smem, std::max(n_max, 1), dmax);
    b->small = need <= (size_t)kSmallSmem;
    b->small_smem = need;
  }
  cudaDeviceProp prop;
  cudaError_t e = cudaGetDeviceProperties(&prop, b->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&b->state, total);
  if (e == cudaSuccess) e = cudaMalloc(&b->inst_d, sizeof(BInst) * n_inst);
  if (e == cudaSuccess) e = set_batch_smem_limit((int)b->smem);
  if (e == cudaSuccess && b->tile_smem) e = set_batch_tile_smem_limit((int)b->tile_smem);
  if (e == cudaSuccess && b->small) e = set_batch_small_smem_limit(kSmallSmem);
  if (e != cudaSuccess) {
    cvq_batch_destroy(b);
    return cuda_err(e, "batch allocation");
  }
  b->sms = prop.multiProcessorCount;
  b->chunks.resize(n_inst);
  for (int i = 0; i < n_inst && b->kind == CVQ_BH; ++i) {
    int nch = 0;
    for (int t = 0; t < b->pv[i].ntypes; ++t) nch = std::max(nch, b->pv[i].types[t].chunk_base + b->pv[i].types[t].nchunks);
    b->chunks[i].resize(nch);
    if (nch) e = cudaMemcpy(b->chunks[i].data(), b->pv[i].P.chunks, sizeof(int4) * nch, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      cvq_batch_destroy(b);
      return cuda_err(e, "copy of the chunk schedules");
    }
  }
  for (int i = 0; i < n_inst; ++i) {
    BInst& I = b->inst[i];
    memset(&I, 0, sizeof I);
    I.S = b->S[i];
    I.P = b->pv[i].P;
    I.ops = b->pv[i].ops_dev;
    char* q = (char*)b->state + offs[i];
    I.psi = (cdf*)q;
    q += a256(sizeof(cdf) * (size_t)I.S.dim);
    I.lam = (cdf*)q;
    q += a256(sizeof(cdf) * (size_t)I.S.dim);
    I.U = (cdf*)q;
    I.ustride = b->pv[i].ustride;
  }
  *out = b;
  return CVQ_OK;
}

extern "C" void cvq_batch_destroy(cvq_batch* b) {
  if (!b) return;
  drop_graph(b);
  drop_screen(b);
  if (b->plan) cudaFree(b->plan);
  if (b->state) cudaFree(b->state);
  if (b->inst_d) cudaFree(b->inst_d);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

extern "C" int cvq_batch_set_ansatz(cvq_batch* b, const int* n_ops, const int* op_ids, const cvq_c128* const* psi0) {
  if (!b || !n_ops || !psi0) return errf(CVQ_EINVAL, "null argument");
  size_t tot = 0;
  for (int i = 0; i < b->n; ++i) {
    if (n_ops[i] < -1 || n_ops[i] > b->n_max) return errf(CVQ_EINVAL, "n_ops[%d] = %d outside [-1, %d]", i, n_ops[i], b->n_max);
    if (n_ops[i] >= 0 && !psi0[i]) return errf(CVQ_EINVAL, "psi0[%d] is NULL", i);
    tot += std::max(n_ops[i], 0);
  }
  if (tot > 0 && !op_ids) return errf(CVQ_EINVAL, "null op_ids");
  size_t o = 0;
  for (int i = 0; i < b->n; ++i)
    for (int k = 0; k < std::max(n_ops[i], 0); ++k, ++o)
      if (op_ids[o] < 0 || op_ids[o] >= b->pv[i].K) return errf(CVQ_EINVAL, "op id %d of instance %d outside its pool", op_ids[o], i);
  b->n_ops.assign(n_ops, n_ops + b->n);
  b->ids.assign(op_ids, op_ids + tot);
  b->psi0.resize(b->n);
  for (int i = 0; i < b->n; ++i) b->psi0[i] = (const double2*)psi0[i];
  return build_plan(b);
}

extern "C" int cvq_batch_set_schedule(cvq_batch* b, int64_t tile, int ctas_per_sm) {
  if (!b) return errf(CVQ_EINVAL, "null argument");
  if (tile < NTHREADS || tile > ((int64_t)1 << 30)) return errf(CVQ_EINVAL, "tile %lld outside [256, 2^30]", (long long)tile);
  if (ctas_per_sm < 1 || ctas_per_sm > 2) return errf(CVQ_EINVAL, "ctas_per_sm must be 1 or 2");
  b->tile = tile;
  b->ctas_per_sm = ctas_per_sm;
  return b->have ? build_plan(b) : CVQ_OK;
}

extern "C" int cvq_batch_energy_and_grad(cvq_batch* b, const double* theta_dev, double* E_dev, double* grad_dev,
                                         void* stream) {
  if (!b || !E_dev) return errf(CVQ_EINVAL, "null argument");
  if (!b->have) return errf(CVQ_EINVAL, "cvq_batch_set_ansatz has not been called");
  if (b->n_theta > 0 && (!theta_dev || !grad_dev)) return errf(CVQ_EINVAL, "null theta / grad");
  if (!b->exec || b->g_theta != theta_dev || b->g_E != E_dev || b->g_grad != grad_dev)
    if (int rc = capture(b, theta_dev, E_dev, grad_dev)) return rc;
  BCUDA(cudaGraphLaunch(b->exec, (cudaStream_t)stream), "graph launch");
  return CVQ_OK;
}

extern "C" int cvq_batch_set_active(cvq_batch* b, const int* active, void* stream) {
  if (!b || !active) return errf(CVQ_EINVAL, "null argument");
  if (!b->have) return errf(CVQ_EINVAL, "cvq_batch_set_ansatz has not been called");
  std::vector<int> a(b->n);
  for (int i = 0; i < b->n; ++i) {
    if (active[i] && b->n_ops[i] < 0) return errf(CVQ_EINVAL, "instance %d has no ansatz", i);
    a[i] = active[i] ? 1 : 0;
  }
  BCUDA(cudaMemcpyAsync(b->active_d, a.data(), sizeof(int) * b->n, cudaMemcpyHostToDevice, (cudaStream_t)stream),
        "copy active flags");
  BCUDA(cudaStreamSynchronize((cudaStream_t)stream), "synchronise");
  return CVQ_OK;
}

extern "C" int cvq_batch_info(const cvq_batch* b, int* kernels_per_eval, int* items, int* layers, int64_t* n_params) {
  if (!b) return errf(CVQ_EINVAL, "null argument");
  int nk = 0;
  for (int n : b->layer_n) nk += n > 0;
  if (kernels_per_eval) *kernels_per_eval = b->small ? 1 + (b->n_gates > 0) : nk + (b->n_gates > 0) + (b->n_red > 0);
  if (items) *items = b->n_items;
  if (layers) *layers = (int)b->layer_n.size();
  if (n_params) *n_params = b->n_theta;
  return CVQ_OK;
}
