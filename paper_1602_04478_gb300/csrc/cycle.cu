// K5: root cycle blocks of length L >= 4 (the DB procedure of Section 5).
//
// The colourful matches of the root cycle C = (a_0 .. a_{L-1}) are split by
// the node a_h that takes the highest data vertex u (Eq. 1).  For each h the
// cycle is cut at a_h and at the opposite node a_d, d = h + floor(L/2), into
// P+ = a_h, a_{h+1}, .., a_d and P- = a_h, a_{h-1}, .., a_d.  A table of
// high-starting matches of each half (every vertex after u lower than u) is
// built by edge extensions (Procedure 1, with NodeJoin / EdgeJoin for the
// annotating blocks, general-cycle figure); P- includes a_h's node block and
// P+ includes a_d's (the endpoint convention of Section 5.2).  Finally the two
// halves are joined at the image x of a_d with signatures overlapping in
// exactly {chi(u), chi(x)} (Procedure 2); their union is the full colour set.
//
// GPU form.  One CTA handles one source u at a time (sources highest first
// from a work counter).  Path levels 1 .. r-1 of each half are pushed into
// dense per-CTA rows indexed by vertex (pair rows: signatures containing
// chi(u) and chi(end)), with touched lists and stamp words instead of
// clearing the arrays.  The last hop of both halves is not stored: for each
// candidate meeting vertex x the CTA pulls the rows of x's lower neighbours,
// forms both halves' tables at x in shared memory and closes the cycle there,
// so the largest level never goes to memory.  Unannotated cycles compute one
// h and multiply by L (rotations map matches with a_h highest onto matches
// with a_0 highest), and their two halves share one chain of levels.
#include <algorithm>

#include "cc_kernels.h"

namespace cc {

constexpr int kCtaThreads = 256;
constexpr int kWarps = kCtaThreads / 32;
constexpr int kMaxLevels = kMaxHalf;

struct CycleScratch {
  char *base = nullptr;
  size_t slot_bytes = 0;
  // offsets inside one slot
  size_t off_stamp = 0;                       // u64 [n]
  size_t off_list[2][kMaxLevels];             // int32 [n] per (half, level)
  size_t off_rows[2][kMaxLevels];             // u64 [n][rstride]
  size_t off_pre[2][kMaxLevels];              // u64 [n][pstride] (node join at that level)
  int rstride[2][kMaxLevels];
  int pstride[2][kMaxLevels];
  size_t off_x = 0;                           // int32 [n] candidate list
  size_t off_counts = 0;                      // int32 [2][kMaxLevels] + 1
  int slots = 0;
  int acc_stride = 0;                         // per-warp accumulator length
  bool shared_chain = false;
  unsigned epoch = 0;                         // launch number, part of every stamp key
};

struct LevelInfo {
  int s_pre, s;
  int node_pos;
  bool join;
  TabU N;
  TabE E;
};

// Length of P+ for highest node h.
__device__ __host__ inline int split_of(const CycleArgs &a, int h) {
  return a.split_h[h] ? a.split_h[h] : (a.split ? a.split : a.L / 2);
}

// Sizes and tables of level j (1..depth) of half `half` for highest node h.
__device__ __host__ inline void level_info(const CycleArgs &a, int h, int half, int j, LevelInfo &out,
                                           int *depth_out) {
  int L = a.L;
  int rp = split_of(a, h), rm = L - rp;
  int depth = half == 0 ? rp : rm;
  if (depth_out) *depth_out = depth;
  int s = half == 0 ? 1 : (a.N[h].p ? a.N[h].s : 1);
  for (int l = 1; l <= j; l++) {
    int pos, epos;
    TabE E;
    if (half == 0) {
      pos = (h + l) % L;
      epos = (h + l - 1) % L;
      E = a.Efw[epos];
    } else {
      pos = (h - l + L) % L;
      E = a.Ebw[pos];
    }
    int s_pre = s + (E.p ? E.s : 2) - 1;
    bool join = (half == 0) ? (a.N[pos].p != nullptr) : (l < depth && a.N[pos].p != nullptr);
    s = s_pre + (join ? a.N[pos].s - 1 : 0);
    if (l == j) {
      out.s_pre = s_pre;
      out.s = s;
      out.node_pos = pos;
      out.join = join;
      out.N = a.N[pos];
      out.E = E;
    }
  }
}

// End of the part of v's row (in graph g) a path from source u may extend
// into: the vertices below u (DB, rows are rank ordered), or the whole row
// (PS and non-root blocks).
__device__ __forceinline__ int64_t row_end(const CycleArgs &a, const GraphView &g, int64_t vb, int32_t v,
                                           int32_t u) {
  return a.no_order ? g.row[v + 1] : lower_bound_i32(g.col, vb, g.row[v + 1], u);
}

// The graph a hop over an edge with table E walks: the data graph, or the
// pair graph of a pair-keyed table (its rows hold the partners x of u).
__device__ __forceinline__ GraphView walk_graph(const CycleArgs &a, const TabE &E) {
  return E.gi >= 0 ? a.pg[E.gi] : a.g;
}

// Row of an edge-keyed table for walk position epos (null: all zero).
__device__ __forceinline__ const u64 *erow_of(const TabE &E, int64_t epos, unsigned long long *status) {
  if (!E.ridx) return E.p + epos * E.R;
  const int64_t r = __ldg(E.ridx + epos);
  if (r >= 0 && E.nrows > 0 && !cc_in(r, E.nrows, status)) return nullptr;
  return r < 0 ? nullptr : E.p + r * E.R;
}

__device__ __forceinline__ int rows_of(int k, int s) {
  // C(k-2, s-2) for the pair rows
  int n = k - 2, r = s - 2;
  if (r < 0 || r > n) return 0;
  int v = 1;
  for (int i = 1; i <= r; i++) v = v * (n - r + i) / i;
  return v;
}

// Stamp words: the high 48 bits hold the key of the (launch, source, h)
// that last touched the vertex, the low 16 bits its level-membership flags,
// so the arrays never need clearing between sources or launches.
// Set flag `bit` of vertex w under key `cur`; true if newly set.
__device__ __forceinline__ bool stamp_set(unsigned long long *stamp, int32_t w, unsigned long long cur, int bit) {
  unsigned long long *p = stamp + w;
  unsigned long long old = *((volatile unsigned long long *)p);
  while (true) {
    unsigned long long nw;
    if ((old >> 16) != cur) nw = (cur << 16) | (1ull << bit);
    else if (old & (1ull << bit)) return false;
    else nw = old | (1ull << bit);
    unsigned long long got = atomicCAS(p, old, nw);
    if (got == old) return true;
    old = got;
  }
}
__device__ __forceinline__ bool stamp_has(const unsigned long long *stamp, int32_t w, unsigned long long cur,
                                          int bit) {
  unsigned long long v = *((const volatile unsigned long long *)(stamp + w));
  return (v >> 16) == cur && (v >> bit & 1ull);
}

// out (pair row of (u, x), size s_in + N.s - 1) += in (pair row (u,x), size s_in) (x) N[x]
__device__ void join_node(const Lut &lut, const u64 *in, int s_in, int R_in, const TabU &N, int32_t x, int cu,
                          int cx, u64 *out, int s_out, unsigned &ovf, int lane, bool atomic_out) {
  const u64 *nrow = N.p + (int64_t)x * N.R;
  for (int j = lane; j < R_in; j += 32) {
    u64 v = in[j];
    if (!v) continue;
    uint32_t m = pmask(lut, s_in, j, cu, cx);
    for (int l = 0; l < N.R; l++) {
      u64 t = __ldg(nrow + l);
      if (!t) continue;
      uint32_t mn = umask(lut, N.s, l, cx);
      if ((m & mn) != (1u << cx)) continue;
      u64 pv = mul_ck(v, t, ovf);
      u64 *dst = out + pslot(lut, m | mn, cu, cx);
      if (atomic_out) atomic_add_ck(dst, pv, ovf);
      else *dst = add_ck(*dst, pv, ovf);
    }
  }
  (void)s_out;
}

// dst (pair row (u, y), size s_in + E.s - 1) += extend(src pair row (u, x) over edge x -> y)
__device__ __forceinline__ void extend_row(const Lut &lut, const u64 *src, int s_in, int R_in, const TabE &E,
                                           int64_t epos, int cu, int cx, int cy, u64 *dst, unsigned &ovf,
                                           unsigned long long *status) {
  if (!E.p) {
    if (cy == cx) return;
    for (int j = 0; j < R_in; j++) {
      u64 v = src[j];
      if (!v) continue;
      uint32_t m = pmask(lut, s_in, j, cu, cx);
      if (m & (1u << cy)) continue;
      atomic_add_ck(dst + pslot(lut, m | (1u << cy), cu, cy), v, ovf);
    }
    return;
  }
  const u64 *erow = erow_of(E, epos, status);
  if (!erow) return;
  for (int l = 0; l < E.R; l++) {
    u64 t = __ldg(erow + l);
    if (!t) continue;
    uint32_t me = pmask(lut, E.s, l, cx, cy);
    for (int j = 0; j < R_in; j++) {
      u64 v = src[j];
      if (!v) continue;
      uint32_t m = pmask(lut, s_in, j, cu, cx);
      if ((m & me) != (1u << cx)) continue;
      atomic_add_ck(dst + pslot(lut, m | me, cu, cy), mul_ck(v, t, ovf), ovf);
    }
  }
}

struct SlotPtrs {
  unsigned long long *stamp;
  int32_t *list[2][kMaxLevels];
  u64 *rows[2][kMaxLevels];
  u64 *pre[2][kMaxLevels];
  int32_t *xlist;
  int *counts;  // [2*kMaxLevels] + x count
};

__device__ SlotPtrs slot_ptrs(const CycleScratch &sc, int slot) {
  SlotPtrs p;
  char *b = sc.base + (size_t)slot * sc.slot_bytes;
  p.stamp = (unsigned long long *)(b + sc.off_stamp);
  for (int hf = 0; hf < 2; hf++)
    for (int l = 0; l < kMaxLevels; l++) {
      p.list[hf][l] = (int32_t *)(b + sc.off_list[hf][l]);
      p.rows[hf][l] = (u64 *)(b + sc.off_rows[hf][l]);
      p.pre[hf][l] = (u64 *)(b + sc.off_pre[hf][l]);
    }
  p.xlist = (int32_t *)(b + sc.off_x);
  p.counts = (int *)(b + sc.off_counts);
  return p;
}

// Last hop w -> x of one half into acc (pair rows (u, x) of P+ or P-): w is
// a vertex of x's row in the hop's graph gg at CSR position e; lv is the
// half's last materialised level (0: the half is the single edge u -> x and
// its start row is {chi(u)}).
__device__ __forceinline__ void pull_hop(const CycleArgs &a, const GraphView &gg, const SlotPtrs &P,
                                         const CycleScratch &sc, unsigned long long cur, int hs, int lv,
                                         const LevelInfo &last, int s_prev, int R_prev, int64_t e, int32_t w,
                                         int cw, int32_t u, int cu, int cx, u64 *acc, unsigned &ovf) {
  // traversal w -> x: its CSR position is rev[e].  A half of one edge (lv
  // 0) is added once per x by edge_hop instead.
  if (lv == 0) return;
  if (!stamp_has(P.stamp, w, cur, hs * kMaxLevels + lv)) return;
  const int64_t ep = last.E.p ? (last.E.use_rev ? e : __ldg(gg.rev + e)) : 0;
  if (last.E.p && !cc_in(ep, gg.nnz, a.status)) return;
  extend_row(a.lut, P.rows[hs][lv] + (int64_t)w * sc.rstride[hs][lv], s_prev, R_prev, last.E, ep, cu, cw, cx, acc,
             ovf, a.status);
}

// P+ of a single edge u -> x (split 1): its row at x, from x's position in
// u's row of the hop's graph (x was found there), added by one lane.
__device__ __forceinline__ void edge_hop(const CycleArgs &a, const GraphView &gg, const LevelInfo &last, int32_t u,
                                         int cu, int32_t x, int cx, u64 *acc, unsigned &ovf) {
  const int64_t ub = gg.row[u], ue = gg.row[u + 1];
  const int64_t q = lower_bound_i32(gg.col, ub, ue, x);
  if (q >= ue || __ldg(gg.col + q) != x) return;
  if (!last.E.p) {
    atomic_add_ck(acc + pslot(a.lut, (1u << cu) | (1u << cx), cu, cx), 1ull, ovf);
    return;
  }
  const int64_t ep = last.E.use_rev ? __ldg(gg.rev + q) : q;
  if (!cc_in(ep, gg.nnz, a.status)) return;
  const u64 *er = erow_of(last.E, ep, a.status);
  if (!er) return;
  for (int l = 0; l < last.E.R; l++) {
    const u64 t = __ldg(er + l);
    if (t) atomic_add_ck(acc + pslot(a.lut, pmask(a.lut, last.E.s, l, cu, cx), cu, cx), t, ovf);
  }
}

// MB: resident CTAs per SM the register allocation is held to.  Launches
// without vertex order (PS, non-root blocks) take 4 (measured: C6 by PS on a
// 10^5-vertex Chung-Lu graph 9.8 s -> 6.1 s), the DB closures 2 (4 was 4-8%
// slower on annotated root cycles).
template <int MB>
__global__ void __launch_bounds__(kCtaThreads, MB) k_cycle(CycleArgs a, CycleScratch sc, int *work_counter) {
  extern __shared__ u64 smem_acc[];
  __shared__ int s_u;
  __shared__ int s_cnt[2 * kMaxLevels + 1];
  __shared__ unsigned long long s_total;
  __shared__ unsigned s_ovf;
  const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
  const int L = a.L, k = a.k;
  const uint32_t K = (1u << k) - 1u;
  SlotPtrs P = slot_ptrs(sc, blockIdx.x);
  u64 *accP = smem_acc + (size_t)wib * 2 * sc.acc_stride;
  u64 *accM = accP + sc.acc_stride;
  // output rows gathered in shared memory: out_mode 1, the current source's
  // row (one per CTA); out_mode 2 and 3, the (u, x) row of each warp
  unsigned long long *obase = smem_acc + (size_t)kWarps * 2 * sc.acc_stride;
  unsigned long long *orow = a.out_mode >= 2 ? obase + (size_t)wib * a.R_out : obase;
  const int o_all = a.out_mode == 0 ? 0 : (a.out_mode == 1 ? a.R_out : kWarps * a.R_out);
  for (int i = tid; i < o_all; i += kCtaThreads) obase[i] = 0;
  unsigned ovf = 0;
  while (true) {
    if (tid == 0) {
      // once a count of this pass has exceeded 2^64-1 the result is fixed
      // (UINT64_MAX, CC_ERR_OVERFLOW): take no further source
      const bool done = *(const volatile unsigned long long *)(a.status + ST_OVERFLOW) != 0ull;
      s_u = done ? -1 : (int)(a.light_end - 1 - atomicAdd(work_counter, 1));
      s_total = 0;
      s_ovf = 0;
    }
    __syncthreads();
    const int32_t u = s_u;
    if (u < 0) break;
    const int cu = a.colors[u];
    bool wrote = false;
    for (int hi = 0; hi < a.n_h; hi++) {
      const int h = a.hs[hi];
      const int rp = split_of(a, h), rm = L - rp;
      const bool key_x = a.out_mode == 1 && a.out_key_x[hi];
      LevelInfo f0, f1;
      level_info(a, h, 0, 1, f0, nullptr);
      level_info(a, h, 1, 1, f1, nullptr);
      // the first hop of each half: u's row (its lower part under DB) in the hop's graph
      const GraphView g0 = walk_graph(a, f0.E), g1 = walk_graph(a, f1.E);
      const int64_t ub0 = g0.row[u], ub1 = g1.row[u];
      const int du0 = a.no_order ? (int)(g0.row[u + 1] - ub0) : g0.lo_cnt[u];
      const int du1 = a.no_order ? (int)(g1.row[u + 1] - ub1) : g1.lo_cnt[u];
      // both halves leave u, over two distinct vertices when they walk one graph
      if (du0 < 1 || du1 < 1 || (g0.row == g1.row && du0 < 2)) continue;
      wrote = true;
      // stamps are cleared after every (source, h), so (u, h) is a unique key
      const unsigned long long cur = ((unsigned long long)(u + 1) << 3) | (unsigned)hi;
      // levels each half materialises; with a shared chain half 0 carries both
      int mat[2] = {rp - 1, rm - 1};
      if (sc.shared_chain) {
        mat[0] = max(rp - 1, rm - 1);
        mat[1] = 0;
      }
      if (tid < 2 * kMaxLevels + 1) s_cnt[tid] = 0;
      __syncthreads();
      // ---- level 1: the first hop of each half ----
      for (int hf = 0; hf < 2; hf++) {
        if (mat[hf] < 1) continue;
        const LevelInfo &li = hf == 0 ? f0 : f1;
        const GraphView &gf = hf == 0 ? g0 : g1;
        const int64_t ub = hf == 0 ? ub0 : ub1;
        const int du = hf == 0 ? du0 : du1;
        for (int i = tid; i < du; i += kCtaThreads) {
          int32_t v = __ldg(gf.col + ub + i);
          if (!cc_in(v, a.g.n, a.status)) v = u;  // (bounds-check build) recorded, then skipped as u's colour
          const int cv = a.colors[v];
          P.list[hf][1][i] = v;
          stamp_set(P.stamp, v, cur, hf * kMaxLevels + 1);
          if (cv == cu) continue;
          u64 *dst = li.join ? P.pre[hf][1] + (int64_t)v * sc.pstride[hf][1]
                             : P.rows[hf][1] + (int64_t)v * sc.rstride[hf][1];
          // start row: source node block (P- only) joined with the first edge
          int s0 = hf == 0 ? 1 : (a.N[h].p ? a.N[h].s : 1);
          const TabE &E = li.E;
          const u64 *erow = nullptr;
          if (E.p) {
            const int64_t ep1 = E.use_rev ? __ldg(gf.rev + ub + i) : ub + i;
            if (!cc_in(ep1, gf.nnz, a.status)) continue;
            erow = erow_of(E, ep1, a.status);
            if (!erow) continue;
          }
          const u64 *nrow = (hf == 1 && a.N[h].p) ? a.N[h].p + (int64_t)u * a.N[h].R : nullptr;
          int n0 = nrow ? a.N[h].R : 1;
          int nE = E.p ? E.R : 1;
          for (int j0 = 0; j0 < n0; j0++) {
            u64 v0 = nrow ? __ldg(nrow + j0) : 1ull;
            if (!v0) continue;
            uint32_t m0 = nrow ? umask(a.lut, s0, j0, cu) : (1u << cu);
            for (int je = 0; je < nE; je++) {
              u64 ve = erow ? __ldg(erow + je) : 1ull;
              if (!ve) continue;
              uint32_t me = E.p ? pmask(a.lut, E.s, je, cu, cv) : ((1u << cu) | (1u << cv));
              if ((m0 & me) != (1u << cu)) continue;
              u64 val = mul_ck(v0, ve, ovf);
              u64 *d = dst + pslot(a.lut, m0 | me, cu, cv);
              *d = add_ck(*d, val, ovf);
            }
          }
        }
        if (tid == 0) s_cnt[hf * kMaxLevels + 1] = du;
      }
      if (a.count_units && tid == 0) {
        // extension out of level 0 for both halves: the first hops times the start row's slots
        u64 r0 = 1 + (u64)(a.N[h].p ? a.N[h].R : 1);
        atomicAdd(a.status + ST_UNITS, (u64)(du0 + du1) / 2 * r0);
        atomicAdd(a.status + ST_SCAN0, (u64)du0 + (u64)du1);
      }
      __syncthreads();
      // node joins at level 1
      for (int hf = 0; hf < 2; hf++) {
        if (mat[hf] < 1) continue;
        const LevelInfo &li = hf == 0 ? f0 : f1;
        if (!li.join) continue;
        const int Rp = rows_of(k, li.s_pre);
        const int du = hf == 0 ? du0 : du1;
        for (int i = wib; i < du; i += kWarps) {
          int32_t v = P.list[hf][1][i];
          join_node(a.lut, P.pre[hf][1] + (int64_t)v * sc.pstride[hf][1], li.s_pre, Rp, li.N, v, cu, a.colors[v],
                    P.rows[hf][1] + (int64_t)v * sc.rstride[hf][1], li.s, ovf, lane, true);
        }
      }
      __syncthreads();
      // ---- pushes: level j -> j+1 ----
      const int maxmat = max(mat[0], mat[1]);
      for (int j = 1; j < maxmat; j++) {
        for (int hf = 0; hf < 2; hf++) {
          if (mat[hf] < j + 1) continue;
          LevelInfo lj, ln;
          level_info(a, h, hf, j, lj, nullptr);
          level_info(a, h, hf, j + 1, ln, nullptr);
          const GraphView gw = walk_graph(a, ln.E);
          const int Rj = rows_of(k, lj.s);
          const int cnt = s_cnt[hf * kMaxLevels + j];
          u64 *dstbase = ln.join ? P.pre[hf][j + 1] : P.rows[hf][j + 1];
          const int dstride = ln.join ? sc.pstride[hf][j + 1] : sc.rstride[hf][j + 1];
          for (int i = wib; i < cnt; i += kWarps) {
            const int32_t v = P.list[hf][j][i];
            const int cv = a.colors[v];
            const u64 *src = P.rows[hf][j] + (int64_t)v * sc.rstride[hf][j];
            const int64_t vb = gw.row[v];
            const int64_t ve = row_end(a, gw, vb, v, u);
            for (int64_t e = vb + lane; e < ve; e += 32) {
              const int32_t w = __ldg(gw.col + e);
              if (!cc_in(w, a.g.n, a.status)) continue;
              if (stamp_set(P.stamp, w, cur, hf * kMaxLevels + j + 1)) {
                int slot = atomicAdd(&s_cnt[hf * kMaxLevels + j + 1], 1);
                P.list[hf][j + 1][slot] = w;
              }
              int64_t epos = ln.E.use_rev ? __ldg(gw.rev + e) : e;
              if (ln.E.p && !cc_in(epos, gw.nnz, a.status)) continue;
              extend_row(a.lut, src, lj.s, Rj, ln.E, epos, cu, cv, a.colors[w], dstbase + (int64_t)w * dstride,
                         ovf, a.status);
            }
          }
        }
        __syncthreads();
        for (int hf = 0; hf < 2; hf++) {
          if (mat[hf] < j + 1) continue;
          LevelInfo ln;
          level_info(a, h, hf, j + 1, ln, nullptr);
          if (!ln.join) continue;
          const int cnt = s_cnt[hf * kMaxLevels + j + 1];
          const int Rp = rows_of(k, ln.s_pre);
          for (int i = wib; i < cnt; i += kWarps) {
            int32_t w = P.list[hf][j + 1][i];
            join_node(a.lut, P.pre[hf][j + 1] + (int64_t)w * sc.pstride[hf][j + 1], ln.s_pre, Rp, ln.N, w, cu,
                      a.colors[w], P.rows[hf][j + 1] + (int64_t)w * sc.rstride[hf][j + 1], ln.s, ovf, lane, true);
          }
        }
        __syncthreads();
      }
      if (a.count_units) {
        for (int hf = 0; hf < 2; hf++) {
          const int depth = hf == 0 ? rp : rm;
          const int hsl = sc.shared_chain ? 0 : hf;
          for (int j = 1; j < depth; j++) {
            LevelInfo lj, ln;
            level_info(a, h, hf, j, lj, nullptr);
            level_info(a, h, hf, j + 1, ln, nullptr);
            const GraphView gw = walk_graph(a, ln.E);
            const u64 Rj = (u64)rows_of(k, lj.s);
            const int cnt = s_cnt[hsl * kMaxLevels + j];
            u64 acc = 0, edges = 0;
            for (int i = tid; i < cnt; i += kCtaThreads) {
              const int32_t v = P.list[hsl][j][i];
              const int64_t vb = gw.row[v];
              const u64 e = (u64)(row_end(a, gw, vb, v, u) - vb);
              acc += e * Rj;
              edges += e;
            }
            if (acc) atomicAdd(a.status + ST_UNITS, acc);
            if (edges && j < 8) atomicAdd(a.status + ST_SCAN0 + j, edges);
          }
        }
      }
      LevelInfo lp_last, lm_last, lp_prev, lm_prev;
      level_info(a, h, 0, rp, lp_last, nullptr);
      level_info(a, h, 1, rm, lm_last, nullptr);
      if (rp > 1) level_info(a, h, 0, rp - 1, lp_prev, nullptr);
      level_info(a, h, 1, rm - 1, lm_prev, nullptr);
      // the last hop of each half walks its own graph
      const GraphView gP = walk_graph(a, lp_last.E), gM = walk_graph(a, lm_last.E);
      // ---- candidate meeting vertices: the last hop out of the smaller last level ----
      int hsrc[2] = {0, sc.shared_chain ? 0 : 1};
      int lsrc[2] = {rp - 1, rm - 1};
      int pick = 0;
      {
        int c0 = lsrc[0] == 0 ? 1 : s_cnt[hsrc[0] * kMaxLevels + lsrc[0]];
        int c1 = s_cnt[hsrc[1] * kMaxLevels + lsrc[1]];
        pick = (c1 < c0) ? 1 : 0;
      }
      {
        const int hf = hsrc[pick], lv = lsrc[pick];
        const GraphView &gc = pick == 0 ? gP : gM;
        const int cnt = lv == 0 ? 1 : s_cnt[hf * kMaxLevels + lv];
        for (int i = wib; i < cnt; i += kWarps) {
          const int32_t v = lv == 0 ? u : P.list[hf][lv][i];
          const int64_t vb = gc.row[v];
          const int64_t ve = row_end(a, gc, vb, v, u);
          for (int64_t e = vb + lane; e < ve; e += 32) {
            const int32_t x = __ldg(gc.col + e);
            if (!cc_in(x, a.g.n, a.status)) continue;
            if (stamp_set(P.stamp, x, cur, 2 * kMaxLevels)) {
              int slot = atomicAdd(&s_cnt[2 * kMaxLevels], 1);
              P.xlist[slot] = x;
            }
          }
        }
      }
      __syncthreads();
      // ---- pull both halves at x and close ----
      {
        const int RPpre = rows_of(k, lp_last.s_pre), RM = rows_of(k, lm_last.s_pre);
        const int sPprev = rp > 1 ? lp_prev.s : 1;
        const int RPprev = rp > 1 ? rows_of(k, lp_prev.s) : 0, RMprev = rows_of(k, lm_prev.s);
        const int xc = s_cnt[2 * kMaxLevels];
        const int hp = hsrc[0], hm = hsrc[1];
        const bool one_walk = gP.row == gM.row;
        u64 mine = 0;
        for (int i = wib; i < xc; i += kWarps) {
          const int32_t x = P.xlist[i];
          const int cx = a.colors[x];
          for (int t = lane; t < RPpre; t += 32) accP[t] = 0;
          for (int t = lane; t < RM; t += 32) accM[t] = 0;
          __syncwarp();
          if (cx != cu) {
            if (rp == 1 && lane == 0) edge_hop(a, gP, lp_last, u, cu, x, cx, accP, ovf);
            const int64_t xb = gP.row[x];
            const int64_t xe = row_end(a, gP, xb, x, u);
            for (int64_t e = xb + lane; e < xe; e += 32) {
              const int32_t w = __ldg(gP.col + e);
              if (!cc_in(w, a.g.n, a.status)) continue;
              const int cw = a.colors[w];
              pull_hop(a, gP, P, sc, cur, hp, rp - 1, lp_last, sPprev, RPprev, e, w, cw, u, cu, cx, accP, ovf);
              if (one_walk)
                pull_hop(a, gM, P, sc, cur, hm, rm - 1, lm_last, lm_prev.s, RMprev, e, w, cw, u, cu, cx, accM, ovf);
            }
            if (!one_walk) {
              const int64_t mb = gM.row[x];
              const int64_t me = row_end(a, gM, mb, x, u);
              for (int64_t e = mb + lane; e < me; e += 32) {
                const int32_t w = __ldg(gM.col + e);
                if (!cc_in(w, a.g.n, a.status)) continue;
                pull_hop(a, gM, P, sc, cur, hm, rm - 1, lm_last, lm_prev.s, RMprev, e, w, a.colors[w], u, cu, cx,
                         accM, ovf);
              }
            }
          }
          __syncwarp();
          if (cx != cu) {
            // closure: (P+ at x, joined with a_d's block) x (P- at x)
            const u64 *nrow = lp_last.join ? lp_last.N.p + (int64_t)x * lp_last.N.R : nullptr;
            const int nN = nrow ? lp_last.N.R : 1;
            for (int t = lane; t < RPpre; t += 32) {
              u64 vp = accP[t];
              if (!vp) continue;
              uint32_t mp = pmask(a.lut, lp_last.s_pre, t, cu, cx);
              for (int l = 0; l < nN; l++) {
                u64 vn = nrow ? __ldg(nrow + l) : 1ull;
                if (!vn) continue;
                uint32_t mn = nrow ? umask(a.lut, lp_last.N.s, l, cx) : (1u << cx);
                if ((mp & mn) != (1u << cx)) continue;
                uint32_t m1 = mp | mn;
                if (a.out_mode) {
                  // non-root block: every P- signature meeting m1 in {chi(u), chi(x)};
                  // the union is the block's signature, counted at u's row
                  // (one boundary node) or at the (u, x) row (two)
                  const u64 vpn = mul_ck(vp, vn, ovf);
                  for (int t2 = 0; t2 < RM; t2++) {
                    const u64 vm = accM[t2];
                    if (!vm) continue;
                    const uint32_t mm = pmask(a.lut, lm_last.s_pre, t2, cu, cx);
                    if ((m1 & mm) != ((1u << cu) | (1u << cx))) continue;
                    const u64 v = mul_ck(vpn, vm, ovf);
                    if (key_x) {
                      // the boundary node is a_d: x's row of the unary table
                      const int slot = uslot(a.lut, m1 | mm, cx);
                      if (!cc_in(slot, a.R_out, a.status)) continue;
                      atomic_add_ck(a.out + (int64_t)x * a.R_out + slot, v, ovf);
                      continue;
                    }
                    const int slot = a.out_mode == 1 ? uslot(a.lut, m1 | mm, cu) : pslot(a.lut, m1 | mm, cu, cx);
                    if (!cc_in(slot, a.R_out, a.status)) continue;
                    const unsigned long long old = atomicAdd(orow + slot, v);
                    ovf |= (old + v < old);
                  }
                  continue;
                }
                uint32_t m2 = (K & ~m1) | (1u << cu) | (1u << cx);
                u64 vm = accM[pslot(a.lut, m2, cu, cx)];
                if (!vm) continue;
                mine = add_ck(mine, mul_ck(mul_ck(vp, vn, ovf), vm, ovf), ovf);
              }
            }
          }
          __syncwarp();
          if (a.out_mode >= 2) {
            // the warp's (u, x) row of a two-boundary block goes out if nonzero
            bool any = false;
            for (int t = lane; t < a.R_out; t += 32) any |= orow[t] != 0ull;
            if (__any_sync(0xffffffffu, any)) {
              int64_t dst = -1;
              if (a.out_mode == 2) {
                // the boundary pair is the edge u -> x of the data graph
                if (lane == 0) {
                  const int64_t q = lower_bound_i32(a.g.col, a.g.row[u], a.g.row[u + 1], x);
                  dst = (q < a.g.row[u + 1] && a.g.col[q] == x) ? q : -1;
                  if (dst < 0) atomicOr(a.status + ST_BADGRAPH, 1ull);
                }
              } else if (lane == 0) {
                const unsigned long long q = atomicAdd(a.pair_count, 1ull);
                if (a.pair_keys) {
                  if ((int64_t)q < a.pair_cap) {
                    a.pair_keys[q] = ((unsigned long long)(uint32_t)u << 32) | (uint32_t)x;
                    dst = (int64_t)q;
                  } else {
                    atomicOr(a.status + ST_PAIRCAP, 1ull);
                  }
                }
              }
              dst = __shfl_sync(0xffffffffu, dst, 0);
              if (dst >= 0) {
                u64 *o = a.out_mode == 2 ? a.out + dst * a.R_out : a.pair_rows + dst * a.R_out;
                for (int t = lane; t < a.R_out; t += 32) o[t] = orow[t];
              }
              for (int t = lane; t < a.R_out; t += 32) orow[t] = 0ull;
            }
            __syncwarp();
          }
        }
        mine = warp_sum_ck(mine, ovf);
        if (lane == 0 && mine) {
          unsigned long long old = atomicAdd(&s_total, mine);
          if (old + mine < old) ovf |= 1u;
        }
      }
      __syncthreads();
      // ---- clear the rows and stamps this source touched (scratch returns to zero) ----
      for (int hf = 0; hf < 2; hf++)
        for (int j = 1; j <= mat[hf]; j++) {
          const int cnt = s_cnt[hf * kMaxLevels + j];
          const int rs = sc.rstride[hf][j], ps = sc.pstride[hf][j];
          for (int i = tid; i < cnt; i += kCtaThreads) {
            int32_t w = P.list[hf][j][i];
            P.list[hf][j][i] = 0;
            u64 *r = P.rows[hf][j] + (int64_t)w * rs;
            for (int t = 0; t < rs; t++) r[t] = 0;
            if (ps) {
              u64 *q = P.pre[hf][j] + (int64_t)w * ps;
              for (int t = 0; t < ps; t++) q[t] = 0;
            }
            P.stamp[w] = 0;
          }
        }
      for (int i = tid; i < s_cnt[2 * kMaxLevels]; i += kCtaThreads) {
        P.stamp[P.xlist[i]] = 0;
        P.xlist[i] = 0;
      }
      __syncthreads();
    }
    if (a.out_mode == 1 && wrote) {
      // u's row of the non-root block's table (only this CTA writes it, or,
      // under DB, other CTAs add to it by atomics too)
      for (int i = tid; i < a.R_out; i += kCtaThreads) {
        if (a.out_atomic) atomic_add_ck(a.out + (int64_t)u * a.R_out + i, orow[i], ovf);
        else a.out[(int64_t)u * a.R_out + i] = orow[i];
        orow[i] = 0;
      }
    }
    if (ovf) atomicOr(&s_ovf, 1u);
    __syncthreads();
    if (tid == 0) {
      unsigned o = s_ovf;
      u64 tot = s_total;
      u64 scaled = tot * (u64)a.multiplier;
      if (a.multiplier > 1 && __umul64hi(tot, (u64)a.multiplier)) o = 1;
      if (a.per_vertex) a.per_vertex[u] = scaled;
      if (scaled) {
        unsigned long long old = atomicAdd(a.status + ST_COUNT, scaled);
        if (old + scaled < old) o = 1;
      }
      if (o) atomicOr(a.status + ST_OVERFLOW, 1ull);
    }
    ovf = 0;
    __syncthreads();
  }
}

static CycleScratch plan_scratch(const CycleArgs &a, int slots) {
  CycleScratch sc;
  int L = a.L, k = a.k;
  bool plain = true;
  for (int i = 0; i < L; i++) plain = plain && !a.N[i].p && !a.Efw[i].p && !a.Ebw[i].p;
  sc.shared_chain = plain;
  for (int hf = 0; hf < 2; hf++)
    for (int l = 0; l < kMaxLevels; l++) sc.rstride[hf][l] = sc.pstride[hf][l] = 0;
  int acc = 1;
  // levels each half materialises, the most over the highest-node choices
  int mat[2] = {0, 0};
  for (int hi = 0; hi < a.n_h; hi++) {
    int h = a.hs[hi];
    const int rp = split_of(a, h), rm = L - rp;
    int mh[2] = {rp - 1, rm - 1};
    if (plain) {
      mh[0] = std::max(rp - 1, rm - 1);
      mh[1] = 0;
    }
    mat[0] = std::max(mat[0], mh[0]);
    mat[1] = std::max(mat[1], mh[1]);
    for (int hf = 0; hf < 2; hf++) {
      for (int l = 1; l <= mh[hf]; l++) {
        LevelInfo li;
        level_info(a, h, hf, l, li, nullptr);
        sc.rstride[hf][l] = std::max<int>(sc.rstride[hf][l], (int)binom(k - 2, li.s - 2));
        if (li.join) sc.pstride[hf][l] = std::max<int>(sc.pstride[hf][l], (int)binom(k - 2, li.s_pre - 2));
      }
      LevelInfo last;
      level_info(a, h, hf, hf == 0 ? rp : rm, last, nullptr);
      acc = std::max<int>(acc, (int)binom(k - 2, last.s_pre - 2));
    }
  }
  sc.acc_stride = acc;
  size_t n = (size_t)a.g.n, off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  sc.off_stamp = take(n * 8);
  for (int hf = 0; hf < 2; hf++)
    for (int l = 0; l < kMaxLevels; l++) {
      bool used = l >= 1 && l <= mat[hf];
      sc.off_list[hf][l] = used ? take(n * 4) : 0;
      sc.off_rows[hf][l] = used ? take(n * 8 * (size_t)sc.rstride[hf][l]) : 0;
      sc.off_pre[hf][l] = (used && sc.pstride[hf][l]) ? take(n * 8 * (size_t)sc.pstride[hf][l]) : 0;
    }
  sc.off_x = take(n * 4);
  sc.off_counts = take(64 * 4);
  sc.slot_bytes = off;
  sc.slots = slots;
  return sc;
}

size_t cycle_scratch_bytes(const CycleArgs &a, int slots) { return plan_scratch(a, slots).slot_bytes * (size_t)slots; }

int launch_cycle(Ctx &c, const CycleArgs &a_in) {
  // triangles come here only without vertex order (pair-keyed tables)
  if (a_in.L < 3 || (a_in.L == 3 && !a_in.no_order) || a_in.L > kMaxCycle) return CC_ERR_UNSUPPORTED;
  if (a_in.split < 0 || a_in.split >= a_in.L || a_in.n_h < 1 || a_in.n_h > a_in.L) return CC_ERR_INVALID_ARG;
  for (int hi = 0; hi < a_in.n_h; hi++) {
    // P- has at least two hops (its first level carries a_h's block); both fit the level arrays
    const int h = a_in.hs[hi];
    if (h < 0 || h >= a_in.L || a_in.split_h[h] < 0 || a_in.split_h[h] >= a_in.L) return CC_ERR_INVALID_ARG;
    const int rp = split_of(a_in, h);
    if (a_in.L - rp < 2) return CC_ERR_INVALID_ARG;
    if (rp > kMaxLevels || a_in.L - rp > kMaxLevels) return CC_ERR_UNSUPPORTED;
  }
  if (a_in.out_mode < 0 || a_in.out_mode > 3 || (a_in.out_mode >= 2 && !a_in.no_order) ||
      (a_in.out_mode == 2 && a_in.split != 1) || (a_in.out_mode == 3 && !a_in.pair_count))
    return CC_ERR_INVALID_ARG;
  CycleArgs a = a_in;
  bool pair_edges = false;
  for (int i = 0; i < a.L; i++) pair_edges = pair_edges || a.Efw[i].gi >= 0 || a.Ebw[i].gi >= 0;
  // sources of degree >= heavy_degree go to the grouped heavy path
  const int64_t n = a.g.n;
  int hd = c.heavy_degree >= 0 ? c.heavy_degree : (c.cur_tuned_heavy >= 0 ? c.cur_tuned_heavy : 256);
  // structural counting, the PS procedure, non-root blocks and pair-keyed
  // tables run on the per-CTA path only
  if (a.count_units || a.no_order || a.out_mode || pair_edges) hd = 1 << 30;
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) / 2;
    if (c.cur_graph_row[mid + 1] - c.cur_graph_row[mid] >= hd) hi = mid;
    else lo = mid + 1;
  }
  a.light_end = (int32_t)lo;
  // plain C4..C6: 16-bit level-2 rows on the heavy path need max degree < 2^16
  // the plain kernels keep 16-bit row entries (degree < 2^16) and tag neighbours with their colour (n < 2^29)
  const bool plain = plain_cycle_eligible(a) && !a.count_units && !a.no_order && (c.cur_graph_row[n] - c.cur_graph_row[n - 1]) < 65536 &&
                     n < ((int64_t)1 << 29);
  if (a.light_end < n) {
    int rc = plain ? run_plain_heavy(c, a, a.light_end) : run_heavy(c, a, a.light_end, heavy_group_size(a));
    if (rc != CC_OK) return rc;
  }
  if (a.light_end == 0) return CC_OK;
  // plain C4..C6 below the threshold: per-CTA push with u32 level-3 rows,
  // exact while max_degree * threshold < 2^32
  if (plain && (double)(c.cur_graph_row[n] - c.cur_graph_row[n - 1]) * (double)hd < 4294967295.0)
    return run_plain_light(c, a, a.light_end);
  CycleScratch one = plan_scratch(a, 1);
  // slots: as many CTAs as memory allows, up to 4 per SM
  size_t budget = c.budget ? (c.budget > c.in_use ? c.budget - c.in_use : 0) : ((size_t)24 << 30);
  size_t per = one.slot_bytes;
  int slots = (int)std::min<size_t>(152 * 4, std::max<size_t>(1, budget / 2 / std::max<size_t>(per, 1)));
  if ((size_t)slots * per > budget && c.budget) return CC_ERR_OOM;
  size_t need = (size_t)slots * per + 256;
  int rc = ensure_scratch(c, need);
  if (rc != CC_OK) return rc;
  CycleScratch sc = plan_scratch(a, slots);
  sc.base = (char *)c.scratch;
  int *counter = (int *)((char *)c.scratch + (size_t)slots * per);
  // rows are cleared by the kernel after each source; a new layout (or a
  // fresh buffer) starts from zeros, and stamp keys carry the launch number
  // every kernel on this scratch returns it to zero, so only a fresh (or
  // failed) buffer needs clearing, whatever layout the previous launch used
  if (c.scratch_dirty) {
    if (cudaMemsetAsync(c.scratch, 0, c.scratch_bytes, c.stream) != cudaSuccess) return CC_ERR_CUDA;
    c.scratch_dirty = false;
  }
  if (cudaMemsetAsync(counter, 0, sizeof(int), c.stream) != cudaSuccess) return CC_ERR_CUDA;
  sc.epoch = 0;
  const size_t o_rows = a.out_mode == 0 ? 0 : (a.out_mode == 1 ? (size_t)a.R_out : (size_t)kWarps * a.R_out);
  size_t smem = (size_t)kWarps * 2 * sc.acc_stride * sizeof(u64) + o_rows * sizeof(u64);
  if (smem > 200 * 1024) return CC_ERR_UNSUPPORTED;
  if (smem > 48 * 1024) {
    cudaFuncSetAttribute(k_cycle<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_cycle<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  // timed apart: root closures, Case-1 blocks, Case-2 blocks
  timing_begin(c, a.out_mode == 0 ? "cycle_closure" : (a.out_mode == 1 ? "cycle_case1" : "cycle_case2"));
  if (a.no_order) k_cycle<4><<<slots, kCtaThreads, smem, c.stream>>>(a, sc, counter);
  else k_cycle<2><<<slots, kCtaThreads, smem, c.stream>>>(a, sc, counter);
  c.kernels++;
  timing_end(c);
  // the queue counter returns to zero too: the whole scratch is zero between launches
  if (cudaMemsetAsync(counter, 0, sizeof(int), c.stream) != cudaSuccess) return CC_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? CC_OK : CC_ERR_CUDA;
}

}  // namespace cc
