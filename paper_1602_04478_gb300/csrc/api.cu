// C-ABI entry points and the plan executor.
//
// The executor walks the decomposition tree bottom-up (Section 4.2, figure
// "Overall Algorithm"): every non-root block gets a projection table --
// unary [n][R] for one boundary node, edge-keyed [nnz][R] for two -- built
// from its children's tables, and the root block is reduced to the count of
// colourful matches.  Tables of a block are freed once its parent has run.
// The estimate is colorful * k^k / k! / aut(Q) (Section 2).
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "cc_kernels.h"

namespace cc {

void *dev_alloc(Ctx &c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (c.budget && c.in_use + bytes > c.budget) return nullptr;
  void *p = nullptr;
  if (c.alloc) {
    p = c.alloc(bytes, c.alloc_user);
  } else if (cudaMallocAsync(&p, bytes, c.stream) != cudaSuccess) {
    // stream-ordered: no device-wide synchronisation, so contexts on other
    // streams keep running while this one allocates
    cudaGetLastError();
    p = nullptr;
  }
  if (p) c.in_use += bytes;
  return p;
}

void dev_free(Ctx &c, void *p, size_t bytes) {
  if (!p) return;
  if (bytes == 0) bytes = 16;
  if (c.free_fn) c.free_fn(p, bytes, c.alloc_user);
  else cudaFreeAsync(p, c.stream);
  c.in_use -= std::min(c.in_use, bytes);
}

int ensure_scratch(Ctx &c, size_t bytes) {
  if (c.scratch_bytes >= bytes) return CC_OK;
  if (c.scratch) {
    cudaStreamSynchronize(c.stream);
    dev_free(c, c.scratch, c.scratch_bytes);
  }
  c.scratch = nullptr;
  c.scratch_bytes = 0;
  c.scratch = dev_alloc(c, bytes);
  if (!c.scratch) return CC_ERR_OOM;
  c.scratch_bytes = bytes;
  c.scratch_dirty = true;
  return CC_OK;
}

int ensure_hv_scratch(Ctx &c, size_t bytes) {
  if (c.hv_scratch_bytes < bytes) {
    if (c.hv_scratch) {
      cudaStreamSynchronize(c.stream);
      dev_free(c, c.hv_scratch, c.hv_scratch_bytes);
    }
    c.hv_scratch = dev_alloc(c, bytes);
    c.hv_scratch_bytes = c.hv_scratch ? bytes : 0;
    if (!c.hv_scratch) return CC_ERR_OOM;
    c.hv_dirty = true;
  }
  if (c.hv_dirty) {
    if (cudaMemsetAsync(c.hv_scratch, 0, c.hv_scratch_bytes, c.stream) != cudaSuccess) return CC_ERR_CUDA;
    c.hv_dirty = false;
  }
  return CC_OK;
}

int ensure_tag_scratch(Ctx &c, size_t bytes) {
  if (c.tag_scratch_bytes >= bytes) return CC_OK;
  if (c.tag_scratch) {
    cudaStreamSynchronize(c.stream);
    dev_free(c, c.tag_scratch, c.tag_scratch_bytes);
  }
  c.tag_scratch = dev_alloc(c, bytes);
  c.tag_scratch_bytes = c.tag_scratch ? bytes : 0;
  return c.tag_scratch ? CC_OK : CC_ERR_OOM;
}

// Every timed stage is also an NVTX range (header-only NVTX 3; a no-op
// unless a profiler listens), whether or not event timing is on.
void timing_begin(Ctx &c, const char *name) {
  nvtxRangePushA(name);
  if (!c.timing) return;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a, c.stream);
  c.pending.push_back({name, {a, b}});
}

void timing_end(Ctx &c) {
  nvtxRangePop();
  if (!c.timing || c.pending.empty()) return;
  cudaEventRecord(c.pending.back().second.second, c.stream);
}

void timing_flush(Ctx &c) {
  if (c.pending.empty()) return;
  cudaStreamSynchronize(c.stream);
  for (auto &p : c.pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.second.first, p.second.second);
    auto &t = c.times[p.first];
    t.first += ms;
    t.second += 1;
    cudaEventDestroy(p.second.first);
    cudaEventDestroy(p.second.second);
  }
  c.pending.clear();
}

namespace {


TabU tab_u(const std::vector<Table> &T, int idx) {
  TabU t;
  if (idx < 0) return t;
  t.p = T[idx].p;
  t.s = T[idx].s;
  t.R = T[idx].R;
  return t;
}
// A pair-keyed table comes back with gi = its stage index; bind_pairs then
// gives it a slot of the cycle's pair graphs (other kernels refuse it).
TabE tab_e(const std::vector<Table> &T, int idx, bool use_rev) {
  TabE t;
  if (idx < 0) return t;
  t.p = T[idx].pair ? T[idx].pg.rows : T[idx].p;
  t.s = T[idx].s;
  t.R = T[idx].R;
  t.use_rev = use_rev;
  if (T[idx].pair) {
    t.gi = idx;
    t.ridx = T[idx].pg.ridx;
    t.nrows = T[idx].pg.n_pairs;
  }
  return t;
}

GraphView pair_view(const PairGraph &pg) {
  GraphView v;
  v.n = pg.n;
  v.nnz = pg.nnz;
  v.row = pg.row;
  v.col = pg.col;
  v.rev = pg.rev;
  v.lo_cnt = pg.lo_cnt;
  return v;
}

// Stage indices in the cycle's edge tables -> slots of a.pg.
int bind_pairs(CycleArgs &a, const std::vector<Table> &T) {
  int used[kMaxPairGraphs], n_used = 0;
  for (int i = 0; i < a.L; i++)
    for (TabE *E : {&a.Efw[i], &a.Ebw[i]}) {
      if (E->gi < 0) continue;
      int slot = -1;
      for (int j = 0; j < n_used; j++)
        if (used[j] == E->gi) slot = j;
      if (slot < 0) {
        if (n_used == kMaxPairGraphs) return CC_ERR_UNSUPPORTED;
        slot = n_used;
        used[n_used++] = E->gi;
        a.pg[slot] = pair_view(T[E->gi].pg);
      }
      E->gi = slot;
    }
  return CC_OK;
}

bool any_pair(const TabE *E, int n) {
  for (int i = 0; i < n; i++)
    if (E[i].gi >= 0) return true;
  return false;
}

size_t table_bytes(const Plan &p, const Stage &st, const DevGraph &g, int *R_out, int *arity) {
  int k = p.k;
  if (st.kind == ST_LEAF || (st.kind == ST_TRI && st.nb == 1) || (st.kind == ST_CYCLE_NONROOT && st.nb == 1)) {
    *arity = 1;
    *R_out = (int)binom(k - 1, st.s - 1);
    return (size_t)g.n * *R_out * 8;
  }
  if ((st.kind == ST_TRI || st.kind == ST_CYCLE_NONROOT) && st.nb == 2) {
    *arity = 2;
    *R_out = (int)binom(k - 2, st.s - 2);
    // a pair-keyed table is sized by its count pass during the pass
    return st.pair_out ? 0 : (size_t)std::max<int64_t>(g.nnz, 1) * *R_out * 8;
  }
  *arity = 0;
  *R_out = 0;
  return 0;
}

int check(cudaError_t e) { return e == cudaSuccess ? CC_OK : CC_ERR_CUDA; }

// Bytes the tables of one colouring pass hold at their peak (all live at once).
size_t plan_table_bytes(const Plan &p, const DevGraph &g) {
  size_t total = 0;
  for (auto &st : p.stages) {
    int R, ar;
    total += table_bytes(p, st, g, &R, &ar);
  }
  return total;
}

}  // namespace

// Bytes one colouring pass of `p` on `g` holds at its peak: every block's
// table (all live at once) and the colouring buffer.
size_t request_table_bytes(const Plan &p, const DevGraph &g) { return plan_table_bytes(p, g) + (size_t)g.n + 256; }

// Device buffers of one colouring pass (PassBuffers): a table per block, the
// colours and the triangle work counter.
int alloc_pass(Ctx &c, const DevGraph &g, const Plan &p, PassBuffers &B) {
  if (c.budget && c.in_use + plan_table_bytes(p, g) + (size_t)g.n + 256 > c.budget) return CC_ERR_OOM;
  B.T.assign(p.stages.size(), Table());
  B.colors = (uint8_t *)dev_alloc(c, (size_t)g.n);
  B.counter = (int *)dev_alloc(c, 256);
  if (!B.colors || !B.counter) return CC_ERR_OOM;
  for (size_t i = 0; i < p.stages.size(); i++) {
    int R = 0, ar = 0;
    size_t bytes = table_bytes(p, p.stages[i], g, &R, &ar);
    B.T[i].arity = ar;
    B.T[i].s = p.stages[i].s;
    B.T[i].R = R;
    if (!bytes) continue;
    B.T[i].p = (u64 *)dev_alloc(c, bytes);
    if (!B.T[i].p) return CC_ERR_OOM;
    B.T[i].bytes = bytes;
    B.T[i].arity = ar;
    B.T[i].s = p.stages[i].s;
    B.T[i].R = R;
  }
  return CC_OK;
}

void free_pass(Ctx &c, const DevGraph &g, PassBuffers &B) {
  for (auto &t : B.T) {
    dev_free(c, t.p, t.bytes);
    if (t.pair) pair_graph_free(c, t.pg);
  }
  B.T.clear();
  dev_free(c, B.colors, (size_t)g.n);
  dev_free(c, B.counter, 256);
  B.colors = nullptr;
  B.counter = nullptr;
}

// Case-2 block of length L >= 4 (two boundary nodes b0 = bd[0], b1 =
// bd[1]): its table cnt(u, x, alpha | B) with u the image of b0 and x that of
// b1, from the general kernel rooted at b0.  The cycle is rotated (and
// reflected if that brings b1 nearer) so that b0 is a_0 and b1 is a_p with
// p <= L/2, and cut at a_0 and a_p: P+ = a_0 .. a_p, P- = a_0, a_{L-1} .. a_p,
// joined at x (Procedure 2 with the cut at the two boundary nodes, no vertex
// order).  A boundary pair joined by a data edge (p = 1) fills the
// edge-keyed table at pos(u -> x); any other pair goes to a pair list --
// counted by one launch, appended by a second into buffers of that size --
// and then into the pair graph a parent walks.  Synchronises (pair lists).
int run_case2(Ctx &c, DevGraph &g, const GraphView &gv, const Lut &lut, const uint8_t *colors, int k,
              const Stage &st, std::vector<Table> &T, size_t i, u64 *status, bool count_units) {
  const int L = st.L;
  int p0 = -1, q0 = -1;
  for (int j = 0; j < L; j++) {
    if (st.nodes[j] == st.bd[0]) p0 = j;
    if (st.nodes[j] == st.bd[1]) q0 = j;
  }
  if (p0 < 0 || q0 < 0) return CC_ERR_INVALID_ARG;
  const int d = (q0 - p0 + L) % L;
  const bool reflect = d > L / 2;
  CycleArgs a;
  a.g = gv;
  a.colors = colors;
  a.k = k;
  a.lut = lut;
  a.L = L;
  for (int j = 0; j < L; j++) {
    if (!reflect) {
      const int o = (j + p0) % L;  // node j is nodes[o]; edge j joins nodes[o] -> nodes[o+1]
      a.N[j] = tab_u(T, st.node_child[o]);
      a.Efw[j] = tab_e(T, st.edge_child[o], !st.edge_fwd[o]);
      a.Ebw[j] = tab_e(T, st.edge_child[o], st.edge_fwd[o]);
    } else {
      const int o = (p0 - j + L) % L;           // node j is nodes[o]
      const int eo = (p0 - j - 1 + 2 * L) % L;  // edge j joins nodes[o] -> nodes[o-1]: edge eo backwards
      a.N[j] = tab_u(T, st.node_child[o]);
      a.Efw[j] = tab_e(T, st.edge_child[eo], st.edge_fwd[eo]);
      a.Ebw[j] = tab_e(T, st.edge_child[eo], !st.edge_fwd[eo]);
    }
  }
  a.split = reflect ? L - d : d;
  a.no_order = true;
  a.n_h = 1;
  a.hs[0] = 0;
  a.multiplier = 1;
  a.per_vertex = nullptr;
  a.status = status;
  a.count_units = count_units;
  a.R_out = T[i].R;
  a.s_out = st.s;
  int rc = bind_pairs(a, T);
  if (rc != CC_OK) return rc;
  if (!st.pair_out) {
    // the boundary pair is the cycle edge a_0 a_1 and a data edge
    if (a.split != 1 || a.Efw[0].gi >= 0 || !T[i].p) return CC_ERR_INVALID_ARG;
    a.out_mode = 2;
    a.out = T[i].p;
    rc = launch_cycle(c, a);
    if (rc != CC_OK) c.scratch_dirty = c.hv_dirty = true;
    return rc;
  }
  // pair list: append into buffers sized from the previous pass of this
  // stage on this graph (the entries vary little between colourings); the
  // launch counts every entry, so one that did not fit is run again into
  // buffers of the exact size.  The first pass only counts.
  if (T[i].pair) pair_graph_free(c, T[i].pg);
  T[i].pair = false;
  unsigned long long *cnt = (unsigned long long *)dev_alloc(c, 16);
  if (!cnt) return CC_ERR_OOM;
  unsigned long long *keys = nullptr;
  u64 *rows = nullptr;
  unsigned long long np = 0;
  int64_t cap = 0;
  const size_t R = (size_t)T[i].R;
  const auto hint_key = std::make_pair((const void *)&st, (int)i);
  auto hint = g.pair_hint.find(hint_key);
  auto alloc_lists = [&](int64_t m) {
    cap = std::max<int64_t>(m, 1);
    keys = (unsigned long long *)dev_alloc(c, (size_t)cap * 8);
    rows = (u64 *)dev_alloc(c, (size_t)cap * R * 8);
    return keys && rows;
  };
  do {
    a.out_mode = 3;
    a.pair_count = cnt;
    if (hint != g.pair_hint.end()) {
      if (!alloc_lists(hint->second + hint->second / 4 + 1024)) { rc = CC_ERR_OOM; break; }
      a.pair_keys = keys;
      a.pair_rows = rows;
      a.pair_cap = cap;
    }
    if ((rc = check(cudaMemsetAsync(cnt, 0, 16, c.stream))) != CC_OK) break;
    if ((rc = launch_cycle(c, a)) != CC_OK) break;
    if ((rc = check(cudaMemcpyAsync(&np, cnt, 8, cudaMemcpyDeviceToHost, c.stream))) != CC_OK) break;
    if ((rc = check(cudaStreamSynchronize(c.stream))) != CC_OK) break;
    if (!keys || (int64_t)np > cap) {
      // counted only, or outgrown: the exact size, and the launch again
      cudaStreamSynchronize(c.stream);
      dev_free(c, keys, (size_t)cap * 8);
      dev_free(c, rows, (size_t)cap * R * 8);
      keys = nullptr;
      rows = nullptr;
      if (!alloc_lists((int64_t)np)) { rc = CC_ERR_OOM; break; }
      a.pair_keys = keys;
      a.pair_rows = rows;
      a.pair_cap = cap;
      a.count_units = false;  // the structural work was counted by the first launch
      // the overflowing launch may have flagged the list's capacity
      if ((rc = check(cudaMemsetAsync(status + ST_PAIRCAP, 0, 8, c.stream))) != CC_OK) break;
      if ((rc = check(cudaMemsetAsync(cnt, 0, 16, c.stream))) != CC_OK) break;
      if ((rc = launch_cycle(c, a)) != CC_OK) break;
    }
    g.pair_hint[hint_key] = (int64_t)np;
    T[i].pg.rows = rows;
    T[i].pg.rows_cap = cap;
    T[i].pg.R = (int)R;
    T[i].pair = true;
    rows = nullptr;  // owned by the pair graph now (freed with the pass)
    rc = pair_graph_build(c, g.n, keys, (int64_t)np, T[i].pg);
  } while (false);
  if (rc != CC_OK) c.scratch_dirty = c.hv_dirty = true;
  cudaStreamSynchronize(c.stream);
  dev_free(c, cnt, 16);
  dev_free(c, keys, (size_t)cap * 8);
  dev_free(c, rows, (size_t)cap * R * 8);
  return rc;
}

bool pair_edges(const Plan &p, const Stage &st) {
  const int ne = st.kind == ST_LEAF ? 1 : (st.kind == ST_ROOT_NODE ? 0 : st.L);
  for (int j = 0; j < ne; j++)
    if (edge_pair_keyed(p.stages, st, j)) return true;
  return false;
}

// A triangle with no or one boundary node that reads a pair-keyed table:
// the cycle kernel with L = 3 and no vertex order (P+ the edge a_0 a_1, P-
// the path a_0 a_2 a_1), rotated so the boundary node is a_0.  Root: every
// colourful match once, by a_0's image; one boundary node: the unary table.
int run_triangle_on_cycle(Ctx &c, const GraphView &gv, const Lut &lut, const uint8_t *colors, int k,
                          const Stage &st, std::vector<Table> &T, size_t i, u64 *status, bool count_units) {
  int p0 = 0;
  if (st.nb == 1)
    while (p0 < 3 && st.nodes[p0] != st.bd[0]) p0++;
  if (p0 == 3) return CC_ERR_INVALID_ARG;
  CycleArgs a;
  a.g = gv;
  a.colors = colors;
  a.k = k;
  a.lut = lut;
  a.L = 3;
  for (int j = 0; j < 3; j++) {
    const int o = (j + p0) % 3;
    a.N[j] = tab_u(T, st.node_child[o]);
    a.Efw[j] = tab_e(T, st.edge_child[o], !st.edge_fwd[o]);
    a.Ebw[j] = tab_e(T, st.edge_child[o], st.edge_fwd[o]);
  }
  a.no_order = true;
  a.n_h = 1;
  a.hs[0] = 0;
  a.multiplier = 1;
  a.per_vertex = nullptr;
  a.status = status;
  a.count_units = count_units;
  if (st.nb == 1) {
    a.out_mode = 1;
    a.out = T[i].p;
    a.R_out = T[i].R;
    a.s_out = st.s;
  }
  int rc = bind_pairs(a, T);
  if (rc != CC_OK) return rc;
  rc = launch_cycle(c, a);
  if (rc != CC_OK) c.scratch_dirty = c.hv_dirty = true;
  return rc;
}

// The block's tables on the cycle in the order a_0 = nodes[p0], a_1, ...
// (reflect: a_0 = nodes[p0], a_1 = nodes[p0 - 1], ...).
void orient_cycle(CycleArgs &a, const Stage &st, const std::vector<Table> &T, int p0, bool reflect) {
  const int L = st.L;
  for (int j = 0; j < L; j++) {
    if (!reflect) {
      const int o = (j + p0) % L;  // node j is nodes[o]; edge j joins nodes[o] -> nodes[o+1]
      a.N[j] = tab_u(T, st.node_child[o]);
      a.Efw[j] = tab_e(T, st.edge_child[o], !st.edge_fwd[o]);
      a.Ebw[j] = tab_e(T, st.edge_child[o], st.edge_fwd[o]);
    } else {
      const int o = (p0 - j + L) % L;           // node j is nodes[o]
      const int eo = (p0 - j - 1 + 2 * L) % L;  // edge j joins nodes[o] -> nodes[o-1]: edge eo backwards
      a.N[j] = tab_u(T, st.node_child[o]);
      a.Efw[j] = tab_e(T, st.edge_child[eo], st.edge_fwd[eo]);
      a.Ebw[j] = tab_e(T, st.edge_child[eo], !st.edge_fwd[eo]);
    }
  }
}

// Case-1 block of length L >= 4 (one boundary node b): its unary table
// cnt(v, alpha | B) by the image v of b.
//   PS: the cycle rotated so b is a_0, one split at a_0 and its opposite
//       node, no vertex order (every image of b a source).
//   DB (Eq. 1 over the block): for each node a_h as the highest, paths below
//       its image u, cut at a_h and at b: for h = b the row is u's; for
//       any other h the cut node b is the meeting vertex x and the row is
//       x's.  The forward distance f from a_h to b sets P+'s length; where f
//       exceeds L/2 the cycle is walked the other way (a second launch with
//       the reflected order), so both halves keep at least two hops.  A cut
//       next to b leaves a half of L - 1 hops, so L <= 6 (longer: PS).
int run_case1(Ctx &c, const GraphView &gv, const Lut &lut, const uint8_t *colors, int k, const Stage &st,
              std::vector<Table> &T, size_t i, u64 *status, bool count_units) {
  const int L = st.L;
  int p0 = 0;
  while (p0 < L && st.nodes[p0] != st.bd[0]) p0++;
  if (p0 == L) return CC_ERR_INVALID_ARG;
  auto base = [&](bool reflect) {
    CycleArgs a;
    a.g = gv;
    a.colors = colors;
    a.k = k;
    a.lut = lut;
    a.L = L;
    orient_cycle(a, st, T, p0, reflect);
    a.multiplier = 1;
    a.per_vertex = nullptr;
    a.status = status;
    a.count_units = count_units;
    a.out_mode = 1;
    a.out = T[i].p;
    a.R_out = T[i].R;
    a.s_out = st.s;
    return a;
  };
  int rc = CC_OK;
  // DB cuts next to b leave a half of L - 1 hops: longer cycles take PS
  if (c.procedure == CC_PROC_PS || L - 1 > kMaxHalf) {
    CycleArgs a = base(false);
    a.no_order = true;
    a.n_h = 1;
    a.hs[0] = 0;
    if ((rc = bind_pairs(a, T)) != CC_OK) return rc;
    rc = launch_cycle(c, a);
    if (rc != CC_OK) c.scratch_dirty = c.hv_dirty = true;
    return rc;
  }
  // DB: h = 0 and the h whose forward distance L - h to b is at most L/2 in
  // this order; the others (1 <= h < L - L/2) reflected, where b lies h ahead
  CycleArgs fw = base(false), bw = base(true);
  fw.no_order = bw.no_order = false;
  fw.out_atomic = bw.out_atomic = true;
  fw.n_h = bw.n_h = 0;
  for (int h = 0; h < L; h++) {
    if (h == 0) {
      fw.hs[fw.n_h++] = 0;  // b highest: u's row, the usual opposite cut
    } else if (L - h <= L / 2) {
      fw.split_h[h] = L - h;
      fw.out_key_x[fw.n_h] = true;
      fw.hs[fw.n_h++] = h;
    } else {
      const int hr = L - h;  // a_h in the reflected order
      bw.split_h[hr] = h;
      bw.out_key_x[bw.n_h] = true;
      bw.hs[bw.n_h++] = hr;
    }
  }
  for (CycleArgs *a : {&fw, &bw}) {
    if (a->n_h == 0) continue;
    if ((rc = bind_pairs(*a, T)) != CC_OK) return rc;
    if ((rc = launch_cycle(c, *a)) != CC_OK) {
      c.scratch_dirty = c.hv_dirty = true;
      return rc;
    }
  }
  return rc;
}

// Issue one colouring pass of the plan on the context's stream: status words
// zeroed, colours, every block bottom-up into its table, the root into
// status[ST_COUNT] (and d_per_vertex, rank order, when given).  No host
// synchronisation, so a sequence of passes can be captured in a CUDA graph.
int enqueue_pass(Ctx &c, DevGraph &g, const Plan &p, int64_t trial, PassBuffers &B, u64 *status,
                 u64 *d_per_vertex, std::vector<StageWork> *detail) {
  const int k = p.k;
  const bool count_units = detail != nullptr;
  int rc = CC_OK;
  if ((rc = check(cudaMemsetAsync(status, 0, (count_units ? kStatusWords : 8) * sizeof(u64), c.stream))) != CC_OK)
    return rc;
  // structural counting: the device counters after the previous stage
  u64 seen[kStatusWords] = {0};
  if ((rc = colors_fill(c, g, k, trial, B.colors)) != CC_OK) return rc;
  if (d_per_vertex && (rc = check(cudaMemsetAsync(d_per_vertex, 0, (size_t)g.n * 8, c.stream))) != CC_OK) return rc;
  Lut lut{c.lut_rank, c.lut_unrank};
  GraphView gv = view_of(g);
  c.cur_graph_row = g.h_row.data();
  c.cur_graph = &g;
  std::vector<Table> &T = B.T;
  for (size_t i = 0; i < p.stages.size() && rc == CC_OK; i++) {
    const Stage &st = p.stages[i];
    bool is_root = i + 1 == p.stages.size();
    const int R = T[i].R;
    if (T[i].p && (rc = check(cudaMemsetAsync(T[i].p, 0, T[i].bytes, c.stream))) != CC_OK) break;
    StageWork w;
    w.kind = st.kind;
    if (st.kind == ST_LEAF) {
      LeafArgs a;
      a.g = gv;
      a.colors = B.colors;
      a.k = k;
      a.lut = lut;
      a.A = tab_u(T, st.node_child[0]);
      a.B = tab_u(T, st.node_child[1]);
      a.E = tab_e(T, st.edge_child[0], !st.edge_fwd[0]);
      u64 *dense = nullptr;
      size_t dense_bytes = 0;
      if (a.E.gi >= 0) {
        // a leaf over a pair-keyed edge walks the pair graph, with the rows
        // laid out by its positions like an edge-keyed table
        const PairGraph &pg = T[a.E.gi].pg;
        dense_bytes = (size_t)std::max<int64_t>(pg.nnz, 1) * pg.R * 8;
        dense = (u64 *)dev_alloc(c, dense_bytes);
        if (!dense) { rc = CC_ERR_OOM; break; }
        if ((rc = pair_rows_by_position(c, pg, dense)) != CC_OK) { dev_free(c, dense, dense_bytes); break; }
        a.g = pair_view(pg);
        a.E.p = dense;
        a.E.ridx = nullptr;
        a.E.gi = -1;
      }
      int sE = a.E.p ? a.E.s : 2, sB = a.B.p ? a.B.s : 1, sA = a.A.p ? a.A.s : 1;
      a.sY = sE + sB - 1;
      a.RY = (int)binom(k - 1, a.sY - 1);
      a.out = T[i].p;
      a.s_out = st.s;
      a.R_out = R;
      a.status = status;
      if (sA + a.sY - 1 != st.s) { rc = CC_ERR_INVALID_ARG; break; }
      // every directed edge joins one edge row with one row of the leaf's
      // block; bytes: one gathered u64 per update, the neighbour id per
      // edge, the A rows read and the output rows written
      w.units = (double)g.nnz * (a.E.p ? a.E.R : 1) * (a.B.p ? a.B.R : 1);
      w.bytes = 8.0 * ((a.E.p || a.B.p) ? w.units : 0.0) + 4.0 * (double)g.nnz +
                8.0 * (double)g.n * ((a.A.p ? a.A.R : 0) + R);
      rc = launch_leaf(c, a);
      dev_free(c, dense, dense_bytes);  // stream-ordered after the join
    } else if (st.kind == ST_TRI && (st.pair_out || pair_edges(p, st))) {
      // a triangle that reads (or writes) a pair-keyed table runs on the
      // cycle kernel without vertex order, cut at a_0 and a_1
      if (st.nb == 2) {
        rc = run_case2(c, g, gv, lut, B.colors, k, st, T, i, status, count_units);
      } else if (is_root && d_per_vertex) {
        rc = CC_ERR_UNSUPPORTED;  // the count would split by a_0's image, not by the highest vertex
      } else {
        rc = run_triangle_on_cycle(c, gv, lut, B.colors, k, st, T, i, status, count_units);
      }
    } else if (st.kind == ST_TRI) {
      TriArgs a;
      a.g = gv;
      a.colors = B.colors;
      a.k = k;
      a.lut = lut;
      for (int j = 0; j < 3; j++) {
        a.N[j] = tab_u(T, st.node_child[j]);
        a.E[j] = tab_e(T, st.edge_child[j], !st.edge_fwd[j]);
      }
      if (any_pair(a.E, 3) || st.pair_out) { rc = CC_ERR_INVALID_ARG; break; }
      a.nb = st.nb;
      for (int b = 0; b < st.nb; b++)
        for (int j = 0; j < 3; j++)
          if (st.nodes[j] == st.bd[b]) a.bd[b] = j;
      a.s_out = st.s;
      a.R_out = R;
      a.out = T[i].p;
      a.per_vertex = is_root ? d_per_vertex : nullptr;
      a.status = status;
      a.work_counter = B.counter;
      a.count_units = count_units;
      rc = launch_triangle(c, a);
      // bytes (completed below from the wedge count): one neighbour id per
      // wedge scanned, the output rows written
      w.bytes = 8.0 * (double)(st.nb == 2 ? g.nnz : (st.nb == 1 ? g.n : 0)) * R;
    } else if (st.kind == ST_CYCLE_ROOT) {
      CycleArgs a;
      a.g = gv;
      a.colors = B.colors;
      a.k = k;
      a.lut = lut;
      a.L = st.L;
      bool plain = true;
      for (int j = 0; j < st.L; j++) {
        a.N[j] = tab_u(T, st.node_child[j]);
        a.Efw[j] = tab_e(T, st.edge_child[j], !st.edge_fwd[j]);
        a.Ebw[j] = tab_e(T, st.edge_child[j], st.edge_fwd[j]);
        plain = plain && st.node_child[j] < 0 && st.edge_child[j] < 0;
      }
      // Rotations of the cycle that carry every annotation onto an identical
      // child subtree map the matches with a_h highest onto those with
      // a_{h+rho} highest: compute h < rho and multiply by L / rho.
      int rho = st.L;
      for (int r = 1; r < st.L; r++) {
        if (st.L % r) continue;
        bool ok = true;
        for (int j = 0; j < st.L && ok; j++) {
          int t = (j + r) % st.L;
          auto sig_of = [&](int child) { return child < 0 ? std::string("-") : p.stages[child].sig; };
          ok = sig_of(st.node_child[j]) == sig_of(st.node_child[t]) &&
               sig_of(st.edge_child[j]) == sig_of(st.edge_child[t]) &&
               (st.edge_child[j] < 0 || st.edge_fwd[j] == st.edge_fwd[t]);
        }
        if (ok) {
          rho = r;
          break;
        }
      }
      (void)plain;
      a.n_h = rho;
      for (int h = 0; h < rho; h++) a.hs[h] = h;
      a.multiplier = st.L / rho;
      if (c.procedure == CC_PROC_PS) {
        // PS: one split (a_0 and its opposite node), no vertex order, every
        // match counted once with a_0's image as the source
        a.no_order = true;
        a.n_h = 1;
        a.hs[0] = 0;
        a.multiplier = 1;
      }
      a.per_vertex = d_per_vertex;
      a.status = status;
      a.count_units = count_units;
      if ((rc = bind_pairs(a, T)) != CC_OK) break;
      rc = launch_cycle(c, a);
      if (rc != CC_OK) c.scratch_dirty = c.hv_dirty = true;
    } else if (st.kind == ST_CYCLE_NONROOT && st.nb == 2) {
      rc = run_case2(c, g, gv, lut, B.colors, k, st, T, i, status, count_units);
    } else if (st.kind == ST_CYCLE_NONROOT && st.nb == 1) {
      rc = run_case1(c, gv, lut, B.colors, k, st, T, i, status, count_units);
    } else if (st.kind == ST_ROOT_NODE) {
      const Table &ct = T[st.node_child[0]];
      if (ct.R != 1) { rc = CC_ERR_INVALID_ARG; break; }
      rc = launch_root_sum(c, gv, ct.p, d_per_vertex, status);
      w.bytes = 8.0 * (double)g.n;
    } else {
      rc = CC_ERR_UNSUPPORTED;
    }
    if (detail && rc == CC_OK) {
      // the device counters this stage added (the pass is not timed or captured)
      u64 now[kStatusWords];
      rc = check(cudaMemcpyAsync(now, status, sizeof(now), cudaMemcpyDeviceToHost, c.stream));
      if (rc == CC_OK) rc = check(cudaStreamSynchronize(c.stream));
      if (rc != CC_OK) break;
      const double dev_units = (double)(now[ST_UNITS] - seen[ST_UNITS]);
      w.units += dev_units;
      if (st.kind == ST_TRI) w.bytes += 4.0 * dev_units;
      if (st.kind == ST_CYCLE_ROOT || st.kind == ST_CYCLE_NONROOT) {
        for (int j = 0; j < 8; j++) {
          w.scans[j] = (double)(now[ST_SCAN0 + j] - seen[ST_SCAN0 + j]);
          w.bytes += 4.0 * w.scans[j];  // one neighbour id per scanned edge
        }
      }
      std::copy(now, now + kStatusWords, seen);
      detail->push_back(w);
    }
  }
  return rc;
}

int status_code(const u64 *st) {
  if (st[ST_BOUNDS]) return CC_ERR_BOUNDS;
  if (st[ST_BADGRAPH]) return CC_ERR_BAD_GRAPH;
  if (st[ST_PAIRCAP]) return CC_ERR_OOM;
  if (st[ST_TIMEOUT] & 1ull) return CC_ERR_TIMEOUT;
  if (st[ST_TIMEOUT] & 2ull) return CC_ERR_UNSUPPORTED;
  if (st[ST_OVERFLOW]) return CC_ERR_OVERFLOW;
  return CC_OK;
}

// One colouring pass (plain form): allocate, enqueue, wait, read the status.
int run_plan(Ctx &c, DevGraph &g, const Plan &p, int64_t trial, u64 *count, bool *overflow,
             u64 *d_per_vertex, std::vector<StageWork> *detail) {
  PassBuffers B;
  int rc = alloc_pass(c, g, p, B);
  if (rc == CC_OK) rc = enqueue_pass(c, g, p, trial, B, c.d_status, d_per_vertex, detail);
  u64 status[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (rc == CC_OK) {
    rc = check(cudaMemcpyAsync(status, c.d_status, sizeof(status), cudaMemcpyDeviceToHost, c.stream));
    if (rc == CC_OK) rc = check(cudaStreamSynchronize(c.stream));
  }
  timing_flush(c);
  cudaStreamSynchronize(c.stream);
  free_pass(c, g, B);
  if (rc != CC_OK) return rc;
  int sc = status_code(status);
  if (sc != CC_OK && sc != CC_ERR_OVERFLOW) return sc;
  *count = status[ST_COUNT];
  *overflow = sc == CC_ERR_OVERFLOW;
  return CC_OK;
}

}  // namespace cc

using namespace cc;

extern "C" {

const char *cc_strerror(int code) {
  switch (code) {
    case CC_OK: return "ok";
    case CC_ERR_INVALID_ARG: return "invalid argument";
    case CC_ERR_BAD_GRAPH: return "graph is not a symmetric simple CSR (self-loop, duplicate or missing reverse edge)";
    case CC_ERR_NOT_TW2: return "query has no block decomposition: treewidth above 2";
    case CC_ERR_K_RANGE: return "query size k outside [2, 12]";
    case CC_ERR_OOM: return "device memory budget exceeded";
    case CC_ERR_OVERFLOW: return "a count exceeded 2^64-1";
    case CC_ERR_TIMEOUT: return "a bounded device wait gave up";
    case CC_ERR_CUDA: return "CUDA runtime error";
    case CC_ERR_UNSUPPORTED: return "query needs a block kind without a kernel (non-root cycle longer than 3 with two boundary nodes, or a cycle longer than 8)";
    case CC_ERR_NOT_CONNECTED: return "query graph is not connected";
    case CC_ERR_BOUNDS: return "an index left its array (bounds-check build)";
    default: return "unknown error";
  }
}

int cc_create(cc_ctx **out, int device, void *cuda_stream) {
  if (!out) return CC_ERR_INVALID_ARG;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) return CC_ERR_CUDA;
  cc_ctx *x = new cc_ctx();
  x->c.device = device;
  x->c.stream = (cudaStream_t)cuda_stream;
  x->c.d_status = (u64 *)dev_alloc(x->c, kStatusWords * sizeof(u64));
  int rc = x->c.d_status ? luts_init(x->c) : CC_ERR_OOM;
  if (rc != CC_OK) {
    cc_destroy(x);
    return rc;
  }
  *out = x;
  return CC_OK;
}

void cc_destroy(cc_ctx *ctx) {
  if (!ctx) return;
  Ctx &c = ctx->c;
  cudaSetDevice(c.device);
  cudaStreamSynchronize(c.stream);
  batch_cache_clear(c);
  for (auto *l : c.lanes) cc_destroy(l);  // batch lanes borrow this context's graphs
  c.lanes.clear();
  for (auto &g : c.graphs) graph_free(c, g.second);
  dev_free(c, c.scratch, c.scratch_bytes);
  dev_free(c, c.hv_scratch, c.hv_scratch_bytes);
  dev_free(c, c.tag_scratch, c.tag_scratch_bytes);
  dev_free(c, c.lut_rank, 4096 * 2);
  dev_free(c, c.lut_unrank, 13 * kUnrankStride * 2);
  dev_free(c, c.d_status, kStatusWords * sizeof(u64));
  // the stream goes last: the frees above are ordered on it
  cudaStreamSynchronize(c.stream);
  if (c.own_stream) {
    if (c.own_stream != c.stream) cudaStreamSynchronize(c.own_stream);
    cudaStreamDestroy(c.own_stream);
  }
  delete ctx;
}

int cc_set_allocator(cc_ctx *ctx, cc_alloc_fn alloc, cc_free_fn free_fn, void *user) {
  if (!ctx || (!alloc) != (!free_fn)) return CC_ERR_INVALID_ARG;
  Ctx &c = ctx->c;
  if (!c.graphs.empty() || c.scratch) return CC_ERR_INVALID_ARG;  // set before any allocation
  // the context's own small buffers move to the new allocator
  cudaStreamSynchronize(c.stream);
  dev_free(c, c.lut_rank, 4096 * 2);
  dev_free(c, c.lut_unrank, 13 * kUnrankStride * 2);
  dev_free(c, c.d_status, kStatusWords * sizeof(u64));
  c.alloc = alloc;
  c.free_fn = free_fn;
  c.alloc_user = user;
  c.d_status = (u64 *)dev_alloc(c, kStatusWords * sizeof(u64));
  if (!c.d_status) return CC_ERR_OOM;
  return luts_init(c);
}

int cc_set_heavy_degree(cc_ctx *ctx, int degree) {
  if (!ctx || degree < -1) return CC_ERR_INVALID_ARG;
  if (ctx->c.heavy_degree != degree) batch_cache_clear(ctx->c);
  ctx->c.heavy_degree = degree;
  return CC_OK;
}

int cc_set_triangle_list(cc_ctx *ctx, int enable) {
  if (!ctx) return CC_ERR_INVALID_ARG;
  if (ctx->c.tri_list != (enable != 0)) batch_cache_clear(ctx->c);
  ctx->c.tri_list = enable != 0;
  return CC_OK;
}

int cc_set_procedure(cc_ctx *ctx, int procedure) {
  if (!ctx || (procedure != CC_PROC_DB && procedure != CC_PROC_PS)) return CC_ERR_INVALID_ARG;
  if (ctx->c.procedure != procedure) batch_cache_clear(ctx->c);
  ctx->c.procedure = procedure;
  return CC_OK;
}

int cc_set_memory_budget(cc_ctx *ctx, size_t bytes) {
  if (!ctx) return CC_ERR_INVALID_ARG;
  ctx->c.budget = bytes;
  return CC_OK;
}

int cc_load_csr(cc_ctx *ctx, int64_t n, const int64_t *row_ptr, const int32_t *col, int64_t nnz,
                int32_t *graph_id) {
  if (!ctx || !graph_id) return CC_ERR_INVALID_ARG;
  Ctx &c = ctx->c;
  cudaSetDevice(c.device);
  DevGraph g;
  int rc = graph_load(c, n, row_ptr, col, nnz, g);
  if (rc != CC_OK) return rc;
  int id = c.next_graph++;
  c.graphs[id] = g;
  *graph_id = id;
  return CC_OK;
}

int cc_free_graph(cc_ctx *ctx, int32_t graph_id) {
  if (!ctx) return CC_ERR_INVALID_ARG;
  auto it = ctx->c.graphs.find(graph_id);
  if (it == ctx->c.graphs.end()) return CC_ERR_INVALID_ARG;
  cudaStreamSynchronize(ctx->c.stream);
  batch_cache_clear(ctx->c);  // cached batches may point into this graph
  graph_free(ctx->c, it->second);
  ctx->c.graphs.erase(it);
  return CC_OK;
}

int cc_graph_info(cc_ctx *ctx, int32_t graph_id, int64_t *n, int64_t *nnz, int64_t *max_degree) {
  if (!ctx) return CC_ERR_INVALID_ARG;
  auto it = ctx->c.graphs.find(graph_id);
  if (it == ctx->c.graphs.end()) return CC_ERR_INVALID_ARG;
  if (n) *n = it->second.n;
  if (nnz) *nnz = it->second.nnz;
  if (max_degree) *max_degree = it->second.max_deg;
  return CC_OK;
}

int cc_set_query(cc_ctx *ctx, int k, int n_edges, const int32_t *edges, int32_t *query_id) {
  if (!ctx || !query_id || n_edges < 0 || (n_edges > 0 && !edges)) return CC_ERR_INVALID_ARG;
  std::vector<std::pair<int, int>> e;
  for (int i = 0; i < n_edges; i++) e.push_back({edges[2 * i], edges[2 * i + 1]});
  Plan p;
  int rc = plan_query(k, e, p);
  if (rc != CC_OK) return rc;
  int id = ctx->c.next_query++;
  ctx->c.plans[id] = p;
  *query_id = id;
  return CC_OK;
}

int cc_set_decomposition(cc_ctx *ctx, int32_t query_id, const int32_t *block_seq, int len) {
  if (ctx) batch_cache_clear(ctx->c);
  if (!ctx || len < 0 || (len > 0 && !block_seq)) return CC_ERR_INVALID_ARG;
  auto it = ctx->c.plans.find(query_id);
  if (it == ctx->c.plans.end()) return CC_ERR_INVALID_ARG;
  std::vector<int> seq(block_seq, block_seq + len);
  Plan p;
  int rc = plan_explicit(it->second.k, it->second.edges, seq, p);
  if (rc != CC_OK) return rc;
  it->second = p;
  for (auto &g : ctx->c.graphs) g.second.work_detail.erase(query_id);
  return CC_OK;
}

int cc_plan_inspect(int k, int n_edges, const int32_t *edges, const int32_t *block_seq, int seq_len, int32_t *out,
                    int cap, int64_t *aut) {
  if (n_edges < 0 || (n_edges > 0 && !edges) || seq_len < 0 || (seq_len > 0 && !block_seq) || cap < 0 ||
      (cap > 0 && !out))
    return CC_ERR_INVALID_ARG;
  std::vector<std::pair<int, int>> e;
  for (int i = 0; i < n_edges; i++) e.push_back({edges[2 * i], edges[2 * i + 1]});
  Plan p;
  int rc = seq_len > 0 ? plan_explicit(k, e, std::vector<int>(block_seq, block_seq + seq_len), p)
                       : plan_query(k, e, p);
  if (rc != CC_OK && rc != CC_ERR_UNSUPPORTED) return rc;
  if (p.stages.empty()) return rc;
  int w = 0;
  auto put = [&](int32_t x) {
    if (w < cap) out[w] = x;
    w++;
  };
  for (auto &st : p.stages) {
    put(st.kind);
    int L = st.kind == ST_ROOT_NODE ? 1 : st.L;
    put(L);
    for (int i = 0; i < L; i++) put(st.nodes[i]);
    put(st.nb);
    for (int i = 0; i < st.nb; i++) put(st.bd[i]);
    std::vector<int> kids;
    int ne = st.kind == ST_LEAF ? 1 : (st.kind == ST_ROOT_NODE ? 0 : L);
    for (int i = 0; i < L; i++)
      if (st.node_child[i] >= 0) kids.push_back(st.node_child[i]);
    for (int i = 0; i < ne; i++)
      if (st.edge_child[i] >= 0) kids.push_back(st.edge_child[i]);
    put((int32_t)kids.size());
    for (int x : kids) put(x);
  }
  if (aut) *aut = p.aut;
  return w;
}

int cc_plan_supported(int k, int n_edges, const int32_t *edges, const int32_t *block_seq, int seq_len) {
  if (n_edges < 0 || (n_edges > 0 && !edges) || seq_len < 0 || (seq_len > 0 && !block_seq)) return CC_ERR_INVALID_ARG;
  std::vector<std::pair<int, int>> e;
  for (int i = 0; i < n_edges; i++) e.push_back({edges[2 * i], edges[2 * i + 1]});
  Plan p;
  int rc = seq_len > 0 ? plan_explicit(k, e, std::vector<int>(block_seq, block_seq + seq_len), p)
                       : plan_query(k, e, p);
  if (rc == CC_ERR_UNSUPPORTED && !p.stages.empty()) return 0;
  return rc == CC_OK ? 1 : rc;
}

int cc_plan_enumerate(int k, int n_edges, const int32_t *edges, int32_t *out, int cap, int *n_plans) {
  if (n_edges < 0 || (n_edges > 0 && !edges) || cap < 0 || (cap > 0 && !out)) return CC_ERR_INVALID_ARG;
  std::vector<std::pair<int, int>> e;
  for (int i = 0; i < n_edges; i++) e.push_back({edges[2 * i], edges[2 * i + 1]});
  std::vector<PlanChoice> plans;
  int rc = plan_enumerate(k, e, plans);
  if (rc != CC_OK) return rc;
  int w = 0;
  auto put = [&](int32_t x) {
    if (w < cap) out[w] = x;
    w++;
  };
  for (auto &p : plans) {
    put((int32_t)p.seq.size());
    put(p.supported);
    put(p.longest);
    put(p.boundary);
    put(p.annotations);
    put(p.is_default);
    put(p.is_paper);
    put((int32_t)std::min(p.cost, 2.0e9));
    for (int x : p.seq) put(x);
  }
  if (n_plans) *n_plans = (int)plans.size();
  return w;
}

int cc_query_info(cc_ctx *ctx, int32_t query_id, int *k, int64_t *aut, int *n_blocks, int *longest_cycle) {
  if (!ctx) return CC_ERR_INVALID_ARG;
  auto it = ctx->c.plans.find(query_id);
  if (it == ctx->c.plans.end()) return CC_ERR_INVALID_ARG;
  if (k) *k = it->second.k;
  if (aut) *aut = it->second.aut;
  if (n_blocks) *n_blocks = (int)it->second.stages.size();
  if (longest_cycle) *longest_cycle = it->second.longest_cycle;
  return CC_OK;
}

int cc_set_coloring_seed(cc_ctx *ctx, uint64_t seed) {
  if (!ctx) return CC_ERR_INVALID_ARG;
  if (ctx->c.seed != seed) batch_cache_clear(ctx->c);  // the seed is baked into captured launches
  ctx->c.seed = seed;
  return CC_OK;
}

int cc_set_colors(cc_ctx *ctx, int32_t graph_id, const uint8_t *colors, int T) {
  if (!ctx || !colors || T <= 0) return CC_ERR_INVALID_ARG;
  batch_cache_clear(ctx->c);
  auto it = ctx->c.graphs.find(graph_id);
  if (it == ctx->c.graphs.end()) return CC_ERR_INVALID_ARG;
  int mx = 0;
  for (int64_t i = 0; i < (int64_t)T * it->second.n; i++) mx = std::max<int>(mx, colors[i]);
  if (mx >= CC_MAX_K) return CC_ERR_INVALID_ARG;
  int rc = colors_set(ctx->c, it->second, colors, T);
  if (rc == CC_OK) it->second.colors_max = mx;
  return rc;
}

int cc_clear_colors(cc_ctx *ctx, int32_t graph_id) {
  if (!ctx) return CC_ERR_INVALID_ARG;
  batch_cache_clear(ctx->c);
  auto it = ctx->c.graphs.find(graph_id);
  if (it == ctx->c.graphs.end()) return CC_ERR_INVALID_ARG;
  return colors_set(ctx->c, it->second, nullptr, 0);
}

static int lookup(cc_ctx *ctx, int32_t graph_id, int32_t query_id, DevGraph **g, Plan **p) {
  if (!ctx) return CC_ERR_INVALID_ARG;
  auto gi = ctx->c.graphs.find(graph_id);
  auto pi = ctx->c.plans.find(query_id);
  if (gi == ctx->c.graphs.end() || pi == ctx->c.plans.end()) return CC_ERR_INVALID_ARG;
  *g = &gi->second;
  *p = &pi->second;
  if (!(*p)->supported) return CC_ERR_UNSUPPORTED;
  // explicit colours must lie in 0..k-1 for this query
  if (gi->second.colors && gi->second.colors_max >= (*p)->k) return CC_ERR_INVALID_ARG;
  return CC_OK;
}

int cc_count(cc_ctx *ctx, int32_t graph_id, int32_t query_id, int first_trial, int T, uint64_t *colorful,
             double *estimate, double *aut) {
  DevGraph *g;
  Plan *p;
  int rc = lookup(ctx, graph_id, query_id, &g, &p);
  if (rc != CC_OK) return rc;
  if (T <= 0 || first_trial < 0 || !colorful) return CC_ERR_INVALID_ARG;
  Ctx &c = ctx->c;
  cudaSetDevice(c.device);
  double scale = 1.0;
  for (int i = 0; i < p->k; i++) scale *= (double)p->k / (double)(i + 1);  // k^k / k!
  int final_rc = CC_OK;
  if ((rc = prepare_plan_graph(c, *g, *p)) != CC_OK) return rc;
  for (int t = 0; t < T; t++) {
    u64 cnt = 0;
    bool ovf = false;
    c.cur_tuned_heavy = g->tuned_heavy.count(query_id) ? g->tuned_heavy[query_id] : -1;
    rc = run_plan(c, *g, *p, (int64_t)first_trial + t, &cnt, &ovf, nullptr, nullptr);
    if (rc != CC_OK) return rc;
    if (ovf) {
      colorful[t] = UINT64_MAX;
      final_rc = CC_ERR_OVERFLOW;
    } else {
      colorful[t] = cnt;
    }
    if (estimate) estimate[t] = ovf ? INFINITY : (double)cnt * scale / (double)p->aut;
  }
  if (aut) *aut = (double)p->aut;
  return final_rc;
}

int cc_count_per_vertex(cc_ctx *ctx, int32_t graph_id, int32_t query_id, int trial, uint64_t *per_vertex,
                        uint64_t *total) {
  DevGraph *g;
  Plan *p;
  int rc = lookup(ctx, graph_id, query_id, &g, &p);
  if (rc != CC_OK) return rc;
  if (!per_vertex || trial < 0) return CC_ERR_INVALID_ARG;
  Ctx &c = ctx->c;
  cudaSetDevice(c.device);
  if ((rc = prepare_plan_graph(c, *g, *p)) != CC_OK) return rc;
  u64 *d_pv = (u64 *)dev_alloc(c, (size_t)g->n * 8);
  if (!d_pv) return CC_ERR_OOM;
  u64 cnt = 0;
  bool ovf = false;
  c.cur_tuned_heavy = g->tuned_heavy.count(query_id) ? g->tuned_heavy[query_id] : -1;
  rc = run_plan(c, *g, *p, trial, &cnt, &ovf, d_pv, nullptr);
  if (rc == CC_OK) {
    std::vector<u64> by_rank(g->n);
    std::vector<int32_t> id_of(g->n);
    if (cudaMemcpy(by_rank.data(), d_pv, g->n * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(id_of.data(), g->id_of, g->n * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
      rc = CC_ERR_CUDA;
    } else {
      for (int64_t r = 0; r < g->n; r++) per_vertex[id_of[r]] = by_rank[r];
      if (total) *total = ovf ? UINT64_MAX : cnt;
      if (ovf) rc = CC_ERR_OVERFLOW;
    }
  }
  dev_free(c, d_pv, (size_t)g->n * 8);
  return rc;
}

// Per-stage structural work of (graph, query), computed once by a counting
// pass (the structure -- reach sets, wedges -- does not depend on the colouring).
static int work_detail(cc_ctx *ctx, int32_t graph_id, int32_t query_id, const std::vector<StageWork> **out) {
  DevGraph *g;
  Plan *p;
  int rc = lookup(ctx, graph_id, query_id, &g, &p);
  if (rc != CC_OK) return rc;
  auto it = g->work_detail.find(query_id);
  if (it == g->work_detail.end()) {
    Ctx &c = ctx->c;
    cudaSetDevice(c.device);
    u64 cnt = 0;
    bool ovf = false;
    std::vector<StageWork> d;
    rc = run_plan(c, *g, *p, 0, &cnt, &ovf, nullptr, &d);
    if (rc != CC_OK) return rc;
    it = g->work_detail.emplace(query_id, d).first;
  }
  *out = &it->second;
  return CC_OK;
}

int cc_work_units(cc_ctx *ctx, int32_t graph_id, int32_t query_id, double *units) {
  if (!units) return CC_ERR_INVALID_ARG;
  const std::vector<StageWork> *d = nullptr;
  int rc = work_detail(ctx, graph_id, query_id, &d);
  if (rc != CC_OK) return rc;
  double w = 0.0;
  for (auto &s : *d) w += s.units;
  *units = w;
  return CC_OK;
}

int cc_work_detail(cc_ctx *ctx, int32_t graph_id, int32_t query_id, int cap, int32_t *kind, double *units,
                   double *alg_bytes, double *scans) {
  if (cap < 0) return CC_ERR_INVALID_ARG;
  const std::vector<StageWork> *d = nullptr;
  int rc = work_detail(ctx, graph_id, query_id, &d);
  if (rc != CC_OK) return rc;
  for (int i = 0; i < cap && i < (int)d->size(); i++) {
    const StageWork &s = (*d)[i];
    if (kind) kind[i] = s.kind;
    if (units) units[i] = s.units;
    if (alg_bytes) alg_bytes[i] = s.bytes;
    if (scans) std::copy(s.scans, s.scans + 8, scans + 8 * i);
  }
  return (int)d->size();
}

int cc_set_timing(cc_ctx *ctx, int enable) {
  if (!ctx) return CC_ERR_INVALID_ARG;
  ctx->c.timing = enable != 0;
  return CC_OK;
}

int cc_get_timing(cc_ctx *ctx, char *names, double *ms, int64_t *launches, int cap) {
  if (!ctx) return CC_ERR_INVALID_ARG;
  timing_flush(ctx->c);
  int i = 0;
  for (auto &t : ctx->c.times) {
    if (i >= cap) break;
    if (names) {
      strncpy(names + 48 * i, t.first.c_str(), 47);
      names[48 * i + 47] = 0;
    }
    if (ms) ms[i] = t.second.first;
    if (launches) launches[i] = t.second.second;
    i++;
  }
  return (int)ctx->c.times.size();
}

int cc_kernel_launches(cc_ctx *ctx, uint64_t *launches) {
  if (!ctx || !launches) return CC_ERR_INVALID_ARG;
  *launches = ctx->c.kernels;
  return CC_OK;
}

int cc_reset_timing(cc_ctx *ctx) {
  if (!ctx) return CC_ERR_INVALID_ARG;
  timing_flush(ctx->c);
  ctx->c.times.clear();
  return CC_OK;
}

}  // extern "C"
