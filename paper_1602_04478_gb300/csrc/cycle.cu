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
constexpr int kMaxLevels = kMaxCycle / 2 + 1;

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

// Sizes and tables of level j (1..depth) of half `half` for highest node h.
__device__ __host__ inline void level_info(const CycleArgs &a, int h, int half, int j, LevelInfo &out,
                                           int *depth_out) {
  int L = a.L;
  int rp = L / 2, rm = L - L / 2;
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

// End of the part of v's row a path from source u may extend into: the
// vertices below u (DB, rows are rank ordered), or the whole row (PS).
__device__ __forceinline__ int64_t row_end(const CycleArgs &a, int64_t vb, int32_t v, int32_t u) {
  return a.no_order ? a.g.row[v + 1] : lower_bound_i32(a.g.col, vb, a.g.row[v + 1], u);
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
                                           int64_t epos, int cu, int cx, int cy, u64 *dst, unsigned &ovf) {
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
  const u64 *erow = E.p + epos * E.R;
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

__global__ void __launch_bounds__(kCtaThreads) k_cycle(CycleArgs a, CycleScratch sc, int *work_counter) {
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
  // unary output (non-root cycle): the current source's row, gathered here
  unsigned long long *orow = smem_acc + (size_t)kWarps * 2 * sc.acc_stride;
  for (int i = tid; i < (a.out ? a.R_out : 0); i += kCtaThreads) orow[i] = 0;
  unsigned ovf = 0;
  const int rp = L / 2, rm = L - L / 2;
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
    const int64_t ub = a.g.row[u];
    // DB: the lower neighbours (a row prefix); PS: every neighbour
    const int du = a.no_order ? (int)(a.g.row[u + 1] - ub) : a.g.lo_cnt[u];
    const int cu = a.colors[u];
    if (du >= 2) {
      for (int hi = 0; hi < a.n_h; hi++) {
        const int h = a.hs[hi];
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
        // ---- level 1: lower neighbours of u ----
        for (int hf = 0; hf < 2; hf++) {
          if (mat[hf] < 1) continue;
          LevelInfo li;
          level_info(a, h, hf, 1, li, nullptr);
          const int Rp = rows_of(k, li.s_pre), R = rows_of(k, li.s);
          for (int i = tid; i < du; i += kCtaThreads) {
            const int32_t v = __ldg(a.g.col + ub + i);
            const int cv = a.colors[v];
            P.list[hf][1][i] = v;
            stamp_set(P.stamp, v, cur, hf * kMaxLevels + 1);
            if (cv == cu) continue;
            u64 *dst = li.join ? P.pre[hf][1] + (int64_t)v * sc.pstride[hf][1]
                               : P.rows[hf][1] + (int64_t)v * sc.rstride[hf][1];
            // start row: source node block (P- only) joined with the first edge
            int s0 = hf == 0 ? 1 : (a.N[h].p ? a.N[h].s : 1);
            const TabE &E = li.E;
            int64_t epos = E.use_rev ? __ldg(a.g.rev + ub + i) : ub + i;
            const u64 *nrow = (hf == 1 && a.N[h].p) ? a.N[h].p + (int64_t)u * a.N[h].R : nullptr;
            int n0 = nrow ? a.N[h].R : 1;
            int nE = E.p ? E.R : 1;
            for (int j0 = 0; j0 < n0; j0++) {
              u64 v0 = nrow ? __ldg(nrow + j0) : 1ull;
              if (!v0) continue;
              uint32_t m0 = nrow ? umask(a.lut, s0, j0, cu) : (1u << cu);
              for (int je = 0; je < nE; je++) {
                u64 ve = E.p ? __ldg(E.p + epos * E.R + je) : 1ull;
                if (!ve) continue;
                uint32_t me = E.p ? pmask(a.lut, E.s, je, cu, cv) : ((1u << cu) | (1u << cv));
                if ((m0 & me) != (1u << cu)) continue;
                u64 val = mul_ck(v0, ve, ovf);
                u64 *d = dst + pslot(a.lut, m0 | me, cu, cv);
                *d = add_ck(*d, val, ovf);
              }
            }
            (void)Rp;
            (void)R;
          }
          if (tid == 0) s_cnt[hf * kMaxLevels + 1] = du;
        }
        if (a.count_units && tid == 0) {
          // extension out of level 0 for both halves: du edges times the start row's slots
          u64 r0 = 1 + (u64)(a.N[h].p ? a.N[h].R : 1);
          atomicAdd(a.status + ST_UNITS, (u64)du * r0);
          atomicAdd(a.status + ST_SCAN0, 2ull * (u64)du);
        }
        __syncthreads();
        // node joins at level 1
        for (int hf = 0; hf < 2; hf++) {
          if (mat[hf] < 1) continue;
          LevelInfo li;
          level_info(a, h, hf, 1, li, nullptr);
          if (!li.join) continue;
          const int Rp = rows_of(k, li.s_pre);
          for (int i = wib; i < du; i += kWarps) {
            int32_t v = P.list[hf][1][i];
            join_node(a.lut, P.pre[hf][1] + (int64_t)v * sc.pstride[hf][1], li.s_pre, Rp, li.N, v, cu,
                      a.colors[v], P.rows[hf][1] + (int64_t)v * sc.rstride[hf][1], li.s, ovf, lane, true);
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
            const int Rj = rows_of(k, lj.s);
            const int cnt = s_cnt[hf * kMaxLevels + j];
            u64 *dstbase = ln.join ? P.pre[hf][j + 1] : P.rows[hf][j + 1];
            const int dstride = ln.join ? sc.pstride[hf][j + 1] : sc.rstride[hf][j + 1];
            for (int i = wib; i < cnt; i += kWarps) {
              const int32_t v = P.list[hf][j][i];
              const int cv = a.colors[v];
              const u64 *src = P.rows[hf][j] + (int64_t)v * sc.rstride[hf][j];
              const int64_t vb = a.g.row[v];
              const int64_t ve = row_end(a, vb, v, u);
              for (int64_t e = vb + lane; e < ve; e += 32) {
                const int32_t w = __ldg(a.g.col + e);
                if (stamp_set(P.stamp, w, cur, hf * kMaxLevels + j + 1)) {
                  int slot = atomicAdd(&s_cnt[hf * kMaxLevels + j + 1], 1);
                  P.list[hf][j + 1][slot] = w;
                }
                int64_t epos = ln.E.use_rev ? __ldg(a.g.rev + e) : e;
                extend_row(a.lut, src, lj.s, Rj, ln.E, epos, cu, cv, a.colors[w],
                           dstbase + (int64_t)w * dstride, ovf);
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
                        a.colors[w], P.rows[hf][j + 1] + (int64_t)w * sc.rstride[hf][j + 1], ln.s, ovf, lane,
                        true);
            }
          }
          __syncthreads();
        }
        if (a.count_units) {
          for (int hf = 0; hf < 2; hf++) {
            const int depth = hf == 0 ? rp : rm;
            const int hsl = sc.shared_chain ? 0 : hf;
            for (int j = 1; j < depth; j++) {
              LevelInfo lj;
              level_info(a, h, hf, j, lj, nullptr);
              const u64 Rj = (u64)rows_of(k, lj.s);
              const int cnt = s_cnt[hsl * kMaxLevels + j];
              u64 acc = 0, edges = 0;
              for (int i = tid; i < cnt; i += kCtaThreads) {
                const int32_t v = P.list[hsl][j][i];
                const int64_t vb = a.g.row[v];
                const u64 e = (u64)(row_end(a, vb, v, u) - vb);
                acc += e * Rj;
                edges += e;
              }
              if (acc) atomicAdd(a.status + ST_UNITS, acc);
              if (edges && j < 8) atomicAdd(a.status + ST_SCAN0 + j, edges);
            }
          }
        }
        // ---- candidate meeting vertices: neighbours (below u) of the smaller last level ----
        int hsrc[2] = {0, sc.shared_chain ? 0 : 1};
        int lsrc[2] = {rp - 1, rm - 1};
        int pick = 0;
        {
          int c0 = s_cnt[hsrc[0] * kMaxLevels + lsrc[0]];
          int c1 = s_cnt[hsrc[1] * kMaxLevels + lsrc[1]];
          pick = (c1 < c0) ? 1 : 0;
        }
        {
          const int hf = hsrc[pick], lv = lsrc[pick];
          const int cnt = s_cnt[hf * kMaxLevels + lv];
          for (int i = wib; i < cnt; i += kWarps) {
            const int32_t v = P.list[hf][lv][i];
            const int64_t vb = a.g.row[v];
            const int64_t ve = row_end(a, vb, v, u);
            for (int64_t e = vb + lane; e < ve; e += 32) {
              const int32_t x = __ldg(a.g.col + e);
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
          LevelInfo lp_last, lm_last, lp_prev, lm_prev;
          level_info(a, h, 0, rp, lp_last, nullptr);
          level_info(a, h, 1, rm, lm_last, nullptr);
          level_info(a, h, 0, rp - 1, lp_prev, nullptr);
          level_info(a, h, 1, rm - 1, lm_prev, nullptr);
          const int RPpre = rows_of(k, lp_last.s_pre), RM = rows_of(k, lm_last.s_pre);
          const int RPprev = rows_of(k, lp_prev.s), RMprev = rows_of(k, lm_prev.s);
          const int xc = s_cnt[2 * kMaxLevels];
          const int hp = hsrc[0], hm = hsrc[1];
          u64 mine = 0;
          for (int i = wib; i < xc; i += kWarps) {
            const int32_t x = P.xlist[i];
            const int cx = a.colors[x];
            for (int t = lane; t < RPpre; t += 32) accP[t] = 0;
            for (int t = lane; t < RM; t += 32) accM[t] = 0;
            __syncwarp();
            if (cx != cu) {
              const int64_t xb = a.g.row[x];
              const int64_t xe = row_end(a, xb, x, u);
              for (int64_t e = xb + lane; e < xe; e += 32) {
                const int32_t w = __ldg(a.g.col + e);
                const int cw = a.colors[w];
                // traversal w -> x: its CSR position is rev[e]
                if (stamp_has(P.stamp, w, cur, hp * kMaxLevels + rp - 1)) {
                  int64_t ep = lp_last.E.p ? (lp_last.E.use_rev ? e : __ldg(a.g.rev + e)) : 0;
                  extend_row(a.lut, P.rows[hp][rp - 1] + (int64_t)w * sc.rstride[hp][rp - 1], lp_prev.s, RPprev,
                             lp_last.E, ep, cu, cw, cx, accP, ovf);
                }
                if (stamp_has(P.stamp, w, cur, hm * kMaxLevels + rm - 1)) {
                  int64_t ep = lm_last.E.p ? (lm_last.E.use_rev ? e : __ldg(a.g.rev + e)) : 0;
                  extend_row(a.lut, P.rows[hm][rm - 1] + (int64_t)w * sc.rstride[hm][rm - 1], lm_prev.s, RMprev,
                             lm_last.E, ep, cu, cw, cx, accM, ovf);
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
                  if (a.out) {
                    // non-root block: every P- signature meeting m1 in {chi(u), chi(x)};
                    // the union is the block's signature, counted at u's row
                    const u64 vpn = mul_ck(vp, vn, ovf);
                    for (int t2 = 0; t2 < RM; t2++) {
                      const u64 vm = accM[t2];
                      if (!vm) continue;
                      const uint32_t mm = pmask(a.lut, lm_last.s_pre, t2, cu, cx);
                      if ((m1 & mm) != ((1u << cu) | (1u << cx))) continue;
                      const u64 v = mul_ck(vpn, vm, ovf);
                      const int slot = uslot(a.lut, m1 | mm, cu);
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
      if (a.out) {
        // u's row of the non-root block's table (only this CTA writes it)
        for (int i = tid; i < a.R_out; i += kCtaThreads) {
          a.out[(int64_t)u * a.R_out + i] = orow[i];
          orow[i] = 0;
        }
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
  int rp = L / 2, rm = L - L / 2;
  bool plain = true;
  for (int i = 0; i < L; i++) plain = plain && !a.N[i].p && !a.Efw[i].p && !a.Ebw[i].p;
  sc.shared_chain = plain;
  int mat[2] = {rp - 1, rm - 1};
  if (plain) {
    mat[0] = std::max(rp - 1, rm - 1);
    mat[1] = 0;
  }
  for (int hf = 0; hf < 2; hf++)
    for (int l = 0; l < kMaxLevels; l++) sc.rstride[hf][l] = sc.pstride[hf][l] = 0;
  int acc = 1;
  for (int hi = 0; hi < a.n_h; hi++) {
    int h = a.hs[hi];
    for (int hf = 0; hf < 2; hf++) {
      for (int l = 1; l <= mat[hf]; l++) {
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
  if (a_in.L < 4 || a_in.L > kMaxCycle) return CC_ERR_UNSUPPORTED;
  CycleArgs a = a_in;
  // sources of degree >= heavy_degree go to the grouped heavy path
  const int64_t n = a.g.n;
  int hd = c.heavy_degree >= 0 ? c.heavy_degree : (c.cur_tuned_heavy >= 0 ? c.cur_tuned_heavy : 256);
  // structural counting and the PS procedure run on the per-CTA path only
  if (a.count_units || a.no_order) hd = 1 << 30;
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
  size_t smem = (size_t)kWarps * 2 * sc.acc_stride * sizeof(u64) + (a.out ? (size_t)a.R_out * sizeof(u64) : 0);
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_cycle, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  timing_begin(c, "cycle_closure");
  k_cycle<<<slots, kCtaThreads, smem, c.stream>>>(a, sc, counter);
  c.kernels++;
  timing_end(c);
  // the queue counter returns to zero too: the whole scratch is zero between launches
  if (cudaMemsetAsync(counter, 0, sizeof(int), c.stream) != cudaSuccess) return CC_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? CC_OK : CC_ERR_CUDA;
}

}  // namespace cc
