// K5, heavy sources: root-cycle closure for the highest-degree sources, a
// group of B sources at a time, each step spread over the whole GPU.
//
// Same procedure as cycle.cu (DB of Section 5: split at the highest node a_h
// and its opposite a_d, build the high-starting halves P+ and P-, join them
// at the image of a_d with signatures overlapping in exactly {chi(u),
// chi(x)}), organised for sources whose paths reach most of the graph:
//   1. level 1 of both halves for the B sources (their lower neighbours);
//   2. pushes level j -> j+1 (atomics into per-source dense rows, touched
//      lists, stamp words), node joins after each push;
//   3. one pull over every candidate meeting vertex x below the group's
//      highest source: x walks its lower neighbours w once, a membership word
//      member[w] says which sources have w in their last stored level, and
//      only those rows are gathered; both halves' tables at x live in
//      per-thread shared-memory accumulators and are closed immediately.
// Vertices are rank-ordered by degree, so neighbouring x in a warp have
// similar list lengths; x of degree >= 32 are handled by a whole warp.
#include <algorithm>

#include "cc_kernels.h"

namespace cc {

constexpr int kHvMaxB = 8;
constexpr int kHvLevels = kMaxCycle / 2 + 1;
constexpr int kHvThreads = 128;

struct HvLevelInfo {
  int s_pre, s;
  bool join;
  TabU N;
  TabE E;
};

// sizes of level j (1..depth) of half `half` for highest node h (same rules as cycle.cu)
__device__ __host__ inline void hv_level(const CycleArgs &a, int h, int half, int j, HvLevelInfo &out) {
  int L = a.L;
  int depth = half == 0 ? L / 2 : L - L / 2;
  int s = half == 0 ? 1 : (a.N[h].p ? a.N[h].s : 1);
  for (int l = 1; l <= j; l++) {
    int pos;
    TabE E;
    if (half == 0) {
      pos = (h + l) % L;
      E = a.Efw[(h + l - 1) % L];
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
      out.join = join;
      out.N = a.N[pos];
      out.E = E;
    }
  }
}

__device__ __host__ inline int hv_rows(int k, int s) {
  int n = k - 2, r = s - 2;
  if (r < 0 || r > n) return 0;
  int v = 1;
  for (int i = 1; i <= r; i++) v = v * (n - r + i) / i;
  return v;
}

struct HvScratch {
  // rows[hf][j]: [B][n][rstride] (node-joined rows); pre: rows before the node join
  u64 *rows[2][kHvLevels];
  u64 *pre[2][kHvLevels];
  int rstride[2][kHvLevels];
  int pstride[2][kHvLevels];
  int32_t *list[2][kHvLevels];  // [B][n]
  int *cnt;                     // [2][kHvLevels][kHvMaxB]
  unsigned long long *stamp;    // [B][n]
  uint32_t *member;             // [n]: bit b P+ last level, bit 8+b P- last level
  u64 *totals;                  // [kHvMaxB]
  int mat[2];                   // stored levels per half (1 .. depth-1)
  int last[2];                  // level each half's last hop starts from
  int lhalf[2];                 // which stored chain each half reads (shared chain: 0)
  bool shared;                  // unannotated cycle: one chain serves both halves
  bool same_acc;                // even-length unannotated cycle: both halves' tables at x are equal
  int accP, accM;               // accumulator lengths
};

struct HvGroup {
  int B;
  int32_t u[kHvMaxB];
  int32_t umax;
  unsigned long long key[kHvMaxB];  // stamp keys
};

__device__ __forceinline__ bool hv_stamp_set(unsigned long long *stamp, int32_t w, unsigned long long cur,
                                             int bit) {
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

// -------------------------------- level 1 --------------------------------
__global__ void k_hv_level1(CycleArgs a, HvScratch S, HvGroup G, int h) {
  if (block_sees_overflow(a.status)) return;  // the result is already UINT64_MAX
  const int64_t n = a.g.n;
  unsigned ovf = 0;
  for (int b = blockIdx.y; b < G.B; b += gridDim.y) {
    const int32_t u = G.u[b];
    const int64_t ub = a.g.row[u];
    const int du = a.g.lo_cnt[u];
    const int cu = a.colors[u];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < du; i += gridDim.x * blockDim.x) {
      const int32_t v = __ldg(a.g.col + ub + i);
      const int cv = a.colors[v];
      for (int hf = 0; hf < 2; hf++) {
        if (S.mat[hf] < 1) continue;
        HvLevelInfo li;
        hv_level(a, h, hf, 1, li);
        S.list[hf][1][(int64_t)b * n + i] = v;
        hv_stamp_set(S.stamp + (int64_t)b * n, v, G.key[b], hf * kHvLevels + 1);
        if (S.last[0] == 1 && S.lhalf[0] == hf) atomicOr(S.member + v, 1u << b);
        if (S.last[1] == 1 && S.lhalf[1] == hf) atomicOr(S.member + v, 1u << (8 + b));
        if (cv == cu) continue;
        u64 *dst = li.join ? S.pre[hf][1] + ((int64_t)b * n + v) * S.pstride[hf][1]
                           : S.rows[hf][1] + ((int64_t)b * n + v) * S.rstride[hf][1];
        const int s0 = hf == 0 ? 1 : (a.N[h].p ? a.N[h].s : 1);
        const TabE &E = li.E;
        const int64_t epos = E.use_rev ? __ldg(a.g.rev + ub + i) : ub + i;
        const u64 *nrow = (hf == 1 && a.N[h].p) ? a.N[h].p + (int64_t)u * a.N[h].R : nullptr;
        const int n0 = nrow ? a.N[h].R : 1, nE = E.p ? E.R : 1;
        for (int j0 = 0; j0 < n0; j0++) {
          u64 v0 = nrow ? __ldg(nrow + j0) : 1ull;
          if (!v0) continue;
          uint32_t m0 = nrow ? umask(a.lut, s0, j0, cu) : (1u << cu);
          for (int je = 0; je < nE; je++) {
            u64 ve = E.p ? __ldg(E.p + epos * E.R + je) : 1ull;
            if (!ve) continue;
            uint32_t me = E.p ? pmask(a.lut, E.s, je, cu, cv) : ((1u << cu) | (1u << cv));
            if ((m0 & me) != (1u << cu)) continue;
            u64 *d = dst + pslot(a.lut, m0 | me, cu, cv);
            *d = add_ck(*d, mul_ck(v0, ve, ovf), ovf);
          }
        }
      }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      for (int hf = 0; hf < 2; hf++) S.cnt[(hf * kHvLevels + 1) * kHvMaxB + b] = S.mat[hf] >= 1 ? du : 0;
    }
  }
  flag_overflow(a.status, ovf);
}

// ------------------------------- node joins -------------------------------
__global__ void k_hv_join(CycleArgs a, HvScratch S, HvGroup G, int h, int hf, int j) {
  if (block_sees_overflow(a.status)) return;  // the result is already UINT64_MAX
  const int64_t n = a.g.n;
  HvLevelInfo li;
  hv_level(a, h, hf, j, li);
  if (!li.join) return;
  const int Rp = hv_rows(a.k, li.s_pre);
  unsigned ovf = 0;
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int b = 0; b < G.B; b++) {
    const int cnt = S.cnt[(hf * kHvLevels + j) * kHvMaxB + b];
    const int cu = a.colors[G.u[b]];
    for (int64_t i = warp0; i < cnt; i += nwarps) {
      const int32_t w = S.list[hf][j][(int64_t)b * n + i];
      const int cw = a.colors[w];
      const u64 *in = S.pre[hf][j] + ((int64_t)b * n + w) * S.pstride[hf][j];
      u64 *out = S.rows[hf][j] + ((int64_t)b * n + w) * S.rstride[hf][j];
      const u64 *nrow = li.N.p + (int64_t)w * li.N.R;
      for (int q = lane; q < Rp; q += 32) {
        u64 v = in[q];
        if (!v) continue;
        uint32_t m = pmask(a.lut, li.s_pre, q, cu, cw);
        for (int l = 0; l < li.N.R; l++) {
          u64 t = __ldg(nrow + l);
          if (!t) continue;
          uint32_t mn = umask(a.lut, li.N.s, l, cw);
          if ((m & mn) != (1u << cw)) continue;
          atomic_add_ck(out + pslot(a.lut, m | mn, cu, cw), mul_ck(v, t, ovf), ovf);
        }
      }
    }
  }
  flag_overflow(a.status, ovf);
}

// --------------------------------- pushes ---------------------------------
__global__ void k_hv_push(CycleArgs a, HvScratch S, HvGroup G, int h, int hf, int j) {
  if (block_sees_overflow(a.status)) return;  // the result is already UINT64_MAX
  const int64_t n = a.g.n;
  HvLevelInfo lj, ln;
  hv_level(a, h, hf, j, lj);
  hv_level(a, h, hf, j + 1, ln);
  const int Rj = hv_rows(a.k, lj.s);
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned ovf = 0;
  u64 *dbase = ln.join ? S.pre[hf][j + 1] : S.rows[hf][j + 1];
  const int dstride = ln.join ? S.pstride[hf][j + 1] : S.rstride[hf][j + 1];
  const bool mark_p = S.last[0] == j + 1 && S.lhalf[0] == hf;
  const bool mark_m = S.last[1] == j + 1 && S.lhalf[1] == hf;
  for (int b = 0; b < G.B; b++) {
    const int32_t u = G.u[b];
    const int cu = a.colors[u];
    const int cnt = S.cnt[(hf * kHvLevels + j) * kHvMaxB + b];
    int *ncnt = S.cnt + (hf * kHvLevels + j + 1) * kHvMaxB + b;
    for (int64_t i = warp0; i < cnt; i += nwarps) {
      const int32_t v = S.list[hf][j][(int64_t)b * n + i];
      const int cv = a.colors[v];
      const u64 *src = S.rows[hf][j] + ((int64_t)b * n + v) * S.rstride[hf][j];
      const int64_t vb = a.g.row[v];
      const int64_t ve = lower_bound_i32(a.g.col, vb, a.g.row[v + 1], u);
      for (int64_t e = vb + lane; e < ve; e += 32) {
        const int32_t w = __ldg(a.g.col + e);
        if (hv_stamp_set(S.stamp + (int64_t)b * n, w, G.key[b], hf * kHvLevels + j + 1)) {
          int slot = atomicAdd(ncnt, 1);
          S.list[hf][j + 1][(int64_t)b * n + slot] = w;
          if (mark_p) atomicOr(S.member + w, 1u << b);
          if (mark_m) atomicOr(S.member + w, 1u << (8 + b));
        }
        const int cw = a.colors[w];
        u64 *dst = dbase + ((int64_t)b * n + w) * dstride;
        if (!ln.E.p) {
          if (cw == cv) continue;
          for (int q = 0; q < Rj; q++) {
            u64 val = src[q];
            if (!val) continue;
            uint32_t m = pmask(a.lut, lj.s, q, cu, cv);
            if (m & (1u << cw)) continue;
            atomic_add_ck(dst + pslot(a.lut, m | (1u << cw), cu, cw), val, ovf);
          }
        } else {
          const int64_t epos = ln.E.use_rev ? __ldg(a.g.rev + e) : e;
          const u64 *erow = ln.E.p + epos * ln.E.R;
          for (int l = 0; l < ln.E.R; l++) {
            u64 t = __ldg(erow + l);
            if (!t) continue;
            uint32_t me = pmask(a.lut, ln.E.s, l, cv, cw);
            for (int q = 0; q < Rj; q++) {
              u64 val = src[q];
              if (!val) continue;
              uint32_t m = pmask(a.lut, lj.s, q, cu, cv);
              if ((m & me) != (1u << cv)) continue;
              atomic_add_ck(dst + pslot(a.lut, m | me, cu, cw), mul_ck(val, t, ovf), ovf);
            }
          }
        }
      }
    }
  }
  flag_overflow(a.status, ovf);
}

// ---------------------------------- pull ----------------------------------
// Extend one stored row of (u, w) over the edge w -> x into acc (pair rows of (u, x)).
__device__ __forceinline__ void hv_extend(const Lut &lut, const u64 *src, int s_in, int R_in, const TabE &E,
                                          int64_t epos, int cu, int cw, int cx, u64 *acc, unsigned &ovf) {
  if (!E.p) {
    for (int q = 0; q < R_in; q++) {
      u64 v = src[q];
      if (!v) continue;
      uint32_t m = pmask(lut, s_in, q, cu, cw);
      if (m & (1u << cx)) continue;
      u64 *d = acc + pslot(lut, m | (1u << cx), cu, cx);
      *d = add_ck(*d, v, ovf);
    }
    return;
  }
  const u64 *erow = E.p + epos * E.R;
  for (int l = 0; l < E.R; l++) {
    u64 t = __ldg(erow + l);
    if (!t) continue;
    uint32_t me = pmask(lut, E.s, l, cw, cx);
    for (int q = 0; q < R_in; q++) {
      u64 v = src[q];
      if (!v) continue;
      uint32_t m = pmask(lut, s_in, q, cu, cw);
      if ((m & me) != (1u << cw)) continue;
      u64 *d = acc + pslot(lut, m | me, cu, cx);
      *d = add_ck(*d, mul_ck(v, t, ovf), ovf);
    }
  }
}

struct HvPullInfo {
  HvLevelInfo pl, ml, pprev, mprev;  // last (pulled) levels and the stored levels they start from
  int RPpre, RM, RPprev, RMprev;
};

// closure at x for source b: (P+ at x joined with a_d's block) x (P- at x)
__device__ __forceinline__ u64 hv_close(const CycleArgs &a, const HvPullInfo &I, const u64 *accP, const u64 *accM,
                                        int32_t x, int cu, int cx, unsigned &ovf) {
  const uint32_t K = (1u << a.k) - 1u;
  const u64 *nrow = I.pl.join ? I.pl.N.p + (int64_t)x * I.pl.N.R : nullptr;
  const int nN = nrow ? I.pl.N.R : 1;
  u64 tot = 0;
  for (int t = 0; t < I.RPpre; t++) {
    u64 vp = accP[t];
    if (!vp) continue;
    uint32_t mp = pmask(a.lut, I.pl.s_pre, t, cu, cx);
    for (int l = 0; l < nN; l++) {
      u64 vn = nrow ? __ldg(nrow + l) : 1ull;
      if (!vn) continue;
      uint32_t mn = nrow ? umask(a.lut, I.pl.N.s, l, cx) : (1u << cx);
      if ((mp & mn) != (1u << cx)) continue;
      uint32_t m2 = (K & ~(mp | mn)) | (1u << cu) | (1u << cx);
      u64 vm = accM[pslot(a.lut, m2, cu, cx)];
      if (!vm) continue;
      tot = add_ck(tot, mul_ck(mul_ck(vp, vn, ovf), vm, ovf), ovf);
    }
  }
  return tot;
}

// accumulate the contributions of neighbours e in [e0, e1) (step de) of x
__device__ __forceinline__ void hv_gather(const CycleArgs &a, const HvScratch &S, const HvGroup &G,
                                          const HvPullInfo &I, int32_t x, int cx, int64_t e0, int64_t e1, int de,
                                          u64 *acc, const int *cuv, unsigned &ovf) {
  const int64_t n = a.g.n;
  const int stride = S.accP + (S.same_acc ? 0 : S.accM);
  for (int64_t e = e0; e < e1; e += de) {
    const int32_t w = __ldg(a.g.col + e);
    uint32_t mem = __ldg(S.member + w);
    if (!mem) continue;
    const int cw = a.colors[w];
    const int64_t rv = __ldg(a.g.rev + e);  // position of w -> x
    for (int b = 0; b < G.B; b++) {
      if (!((mem >> b) & 0x101u)) continue;
      if (x >= G.u[b] || w >= G.u[b]) continue;
      const int cu = cuv[b];
      if (cu == cx || cw == cx) continue;
      u64 *aP = acc + b * stride;
      if ((mem >> b) & 1u) {
        const int lh = S.lhalf[0], lv = S.last[0];
        int64_t ep = I.pl.E.p ? (I.pl.E.use_rev ? e : rv) : 0;
        hv_extend(a.lut, S.rows[lh][lv] + ((int64_t)b * n + w) * S.rstride[lh][lv], I.pprev.s, I.RPprev, I.pl.E,
                  ep, cu, cw, cx, aP, ovf);
      }
      if (!S.same_acc && ((mem >> (8 + b)) & 1u)) {
        const int lh = S.lhalf[1], lv = S.last[1];
        int64_t ep = I.ml.E.p ? (I.ml.E.use_rev ? e : rv) : 0;
        hv_extend(a.lut, S.rows[lh][lv] + ((int64_t)b * n + w) * S.rstride[lh][lv], I.mprev.s, I.RMprev, I.ml.E,
                  ep, cu, cw, cx, aP + S.accP, ovf);
      }
    }
  }
}

__global__ void __launch_bounds__(kHvThreads) k_hv_pull(CycleArgs a, HvScratch S, HvGroup G, int h,
                                                        int32_t x_split) {
  if (block_sees_overflow(a.status)) return;  // the result is already UINT64_MAX
  extern __shared__ u64 hv_acc[];
  const int tid = threadIdx.x, lane = tid & 31;
  const int stride = S.accP + (S.same_acc ? 0 : S.accM);
  const int per_thread = G.B * stride;
  u64 *acc = hv_acc + (size_t)tid * per_thread;
  HvPullInfo I;
  const int rp = a.L / 2, rm = a.L - a.L / 2;
  hv_level(a, h, 0, rp, I.pl);
  hv_level(a, h, 1, rm, I.ml);
  hv_level(a, h, 0, rp - 1, I.pprev);
  hv_level(a, h, 1, rm - 1, I.mprev);
  I.RPpre = hv_rows(a.k, I.pl.s_pre);
  I.RM = hv_rows(a.k, I.ml.s_pre);
  I.RPprev = hv_rows(a.k, I.pprev.s);
  I.RMprev = hv_rows(a.k, I.mprev.s);
  int cuv[kHvMaxB];
  for (int b = 0; b < kHvMaxB; b++) cuv[b] = b < G.B ? a.colors[G.u[b]] : 0;
  u64 tot[kHvMaxB];
  for (int b = 0; b < kHvMaxB; b++) tot[b] = 0;
  unsigned ovf = 0;
  // low-degree meeting vertices: one thread each
  const int32_t lo_end = min(x_split, G.umax);
  for (int32_t x = blockIdx.x * blockDim.x + tid; x < lo_end; x += gridDim.x * blockDim.x) {
    const int64_t xb = a.g.row[x];
    const int64_t xe = lower_bound_i32(a.g.col, xb, a.g.row[x + 1], G.umax);
    // which sources have a stored-level vertex among x's neighbours at all
    uint32_t any = 0;
    for (int64_t e = xb; e < xe; e++) any |= __ldg(S.member + __ldg(a.g.col + e));
    any = (any | (any >> 8)) & ((1u << G.B) - 1u);
    if (!any) continue;
    const int cx = a.colors[x];
    for (int b = 0; b < G.B; b++)
      if ((any >> b) & 1u)
        for (int q = 0; q < stride; q++) acc[b * stride + q] = 0;
    hv_gather(a, S, G, I, x, cx, xb, xe, 1, acc, cuv, ovf);
    for (int b = 0; b < G.B; b++) {
      if (!((any >> b) & 1u)) continue;
      if (x >= G.u[b] || cx == cuv[b]) continue;
      const u64 *aP = acc + b * stride;
      tot[b] = add_ck(tot[b], hv_close(a, I, aP, S.same_acc ? aP : aP + S.accP, x, cuv[b], cx, ovf), ovf);
    }
  }
  // high-degree meeting vertices: one warp each, lanes split the neighbours
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + tid) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t xi = (int64_t)x_split + warp0; xi < G.umax; xi += nwarps) {
    const int32_t x = (int32_t)xi;
    const int cx = a.colors[x];
    const int64_t xb = a.g.row[x];
    const int64_t xe = lower_bound_i32(a.g.col, xb, a.g.row[x + 1], G.umax);
    uint32_t any = 0;
    for (int64_t e = xb + lane; e < xe; e += 32) any |= __ldg(S.member + __ldg(a.g.col + e));
    any = __reduce_or_sync(0xffffffffu, any);
    any = (any | (any >> 8)) & ((1u << G.B) - 1u);
    if (!any) continue;
    for (int q = 0; q < per_thread; q++) acc[q] = 0;
    hv_gather(a, S, G, I, x, cx, xb + lane, xe, 32, acc, cuv, ovf);
    __syncwarp();
    // sum the 32 lanes' accumulators into lane 0's (slot-parallel)
    u64 *base = hv_acc + (size_t)(tid & ~31) * per_thread;
    for (int q = lane; q < per_thread; q += 32) {
      u64 s = 0;
      for (int l = 0; l < 32; l++) s = add_ck(s, base[(size_t)l * per_thread + q], ovf);
      base[q] = s;
    }
    __syncwarp();
    if (lane == 0) {
      for (int b = 0; b < G.B; b++) {
        if (!((any >> b) & 1u)) continue;
        if (x >= G.u[b] || cx == cuv[b]) continue;
        const u64 *aP = base + b * stride;
        tot[b] = add_ck(tot[b], hv_close(a, I, aP, S.same_acc ? aP : aP + S.accP, x, cuv[b], cx, ovf), ovf);
      }
    }
    __syncwarp();
  }
  for (int b = 0; b < G.B; b++) {
    u64 t = warp_sum_ck(tot[b], ovf);
    if (lane == 0 && t) atomic_add_ck(S.totals + b, t, ovf);
  }
  flag_overflow(a.status, ovf);
}

// --------------------------------- clearing ---------------------------------
__global__ void k_hv_clear(CycleArgs a, HvScratch S, HvGroup G) {
  const int64_t n = a.g.n;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nt = (int64_t)gridDim.x * blockDim.x;
  for (int hf = 0; hf < 2; hf++)
    for (int j = 1; j <= S.mat[hf]; j++)
      for (int b = 0; b < G.B; b++) {
        const int cnt = S.cnt[(hf * kHvLevels + j) * kHvMaxB + b];
        const int rs = S.rstride[hf][j], ps = S.pstride[hf][j];
        for (int64_t i = t0; i < cnt; i += nt) {
          const int32_t w = S.list[hf][j][(int64_t)b * n + i];
          S.list[hf][j][(int64_t)b * n + i] = 0;
          u64 *r = S.rows[hf][j] + ((int64_t)b * n + w) * rs;
          for (int q = 0; q < rs; q++) r[q] = 0;
          if (ps) {
            u64 *p = S.pre[hf][j] + ((int64_t)b * n + w) * ps;
            for (int q = 0; q < ps; q++) p[q] = 0;
          }
          S.member[w] = 0;
          S.stamp[(int64_t)b * n + w] = 0;
        }
      }
}

__global__ void k_hv_finish(CycleArgs a, HvScratch S, HvGroup G, int last_h) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  unsigned ovf = 0;
  for (int b = 0; b < G.B; b++) {
    u64 t = S.totals[b];
    S.totals[b] = 0;
    if (!last_h) {
      S.totals[kHvMaxB + b] = add_ck(S.totals[kHvMaxB + b], t, ovf);
      continue;
    }
    t = add_ck(t, S.totals[kHvMaxB + b], ovf);
    S.totals[kHvMaxB + b] = 0;
    u64 scaled = mul_ck(t, (u64)a.multiplier, ovf);
    if (a.per_vertex) a.per_vertex[G.u[b]] = scaled;
    atomic_add_ck(a.status + ST_COUNT, scaled, ovf);
  }
  flag_overflow(a.status, ovf);
}

// ------------------------------ orchestration ------------------------------
int heavy_group_size(const CycleArgs &a) {
  int rp = a.L / 2, rm = a.L - a.L / 2;
  int worst = 1;
  for (int hi = 0; hi < a.n_h; hi++) {
    HvLevelInfo pl, ml;
    hv_level(a, a.hs[hi], 0, rp, pl);
    hv_level(a, a.hs[hi], 1, rm, ml);
    worst = std::max(worst, hv_rows(a.k, pl.s_pre) + hv_rows(a.k, ml.s_pre));
  }
  int B = 96 / worst;
  return std::max(1, std::min(kHvMaxB, B));
}

int run_heavy(Ctx &c, const CycleArgs &a, int32_t first_rank, int B) {
  const int64_t n = a.g.n;
  if (first_rank >= n) return CC_OK;
  const int rp = a.L / 2, rm = a.L - a.L / 2;
  bool plain = true;
  for (int i = 0; i < a.L; i++) plain = plain && !a.N[i].p && !a.Efw[i].p && !a.Ebw[i].p;
  HvScratch S;
  S.shared = plain;
  S.same_acc = plain && (a.L % 2 == 0);
  S.mat[0] = rp - 1;
  S.mat[1] = rm - 1;
  if (plain) {
    S.mat[0] = std::max(rp - 1, rm - 1);
    S.mat[1] = 0;
  }
  S.last[0] = rp - 1;
  S.last[1] = rm - 1;
  S.lhalf[0] = 0;
  S.lhalf[1] = plain ? 0 : 1;
  int accP = 1, accM = 1;
  for (int hf = 0; hf < 2; hf++)
    for (int l = 0; l < kHvLevels; l++) S.rstride[hf][l] = S.pstride[hf][l] = 0;
  for (int hi = 0; hi < a.n_h; hi++) {
    int h = a.hs[hi];
    for (int hf = 0; hf < 2; hf++)
      for (int l = 1; l <= S.mat[hf]; l++) {
        HvLevelInfo li;
        hv_level(a, h, hf, l, li);
        S.rstride[hf][l] = std::max(S.rstride[hf][l], hv_rows(a.k, li.s));
        if (li.join) S.pstride[hf][l] = std::max(S.pstride[hf][l], hv_rows(a.k, li.s_pre));
      }
    HvLevelInfo pl, ml;
    hv_level(a, h, 0, rp, pl);
    hv_level(a, h, 1, rm, ml);
    accP = std::max(accP, hv_rows(a.k, pl.s_pre));
    accM = std::max(accM, hv_rows(a.k, ml.s_pre));
  }
  S.accP = accP;
  S.accM = accM;
  // scratch layout
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  size_t o_rows[2][kHvLevels], o_pre[2][kHvLevels], o_list[2][kHvLevels];
  for (int hf = 0; hf < 2; hf++)
    for (int l = 0; l < kHvLevels; l++) {
      bool used = l >= 1 && l <= S.mat[hf];
      o_rows[hf][l] = used ? take((size_t)B * n * S.rstride[hf][l] * 8) : 0;
      o_pre[hf][l] = (used && S.pstride[hf][l]) ? take((size_t)B * n * S.pstride[hf][l] * 8) : 0;
      o_list[hf][l] = used ? take((size_t)B * n * 4) : 0;
    }
  size_t o_cnt = take(2 * kHvLevels * kHvMaxB * sizeof(int));
  size_t o_stamp = take((size_t)B * n * 8);
  size_t o_member = take((size_t)n * 4);
  size_t o_tot = take(2 * kHvMaxB * 8);
  size_t need = off;
  int rc0 = ensure_hv_scratch(c, need);
  if (rc0 != CC_OK) return rc0;
  char *base = (char *)c.hv_scratch;
  for (int hf = 0; hf < 2; hf++)
    for (int l = 0; l < kHvLevels; l++) {
      S.rows[hf][l] = (u64 *)(base + o_rows[hf][l]);
      S.pre[hf][l] = (u64 *)(base + o_pre[hf][l]);
      S.list[hf][l] = (int32_t *)(base + o_list[hf][l]);
    }
  S.cnt = (int *)(base + o_cnt);
  S.stamp = (unsigned long long *)(base + o_stamp);
  S.member = (uint32_t *)(base + o_member);
  S.totals = (u64 *)(base + o_tot);
  size_t smem = (size_t)kHvThreads * B * (S.accP + (S.same_acc ? 0 : S.accM)) * 8;
  if (smem > 200 * 1024) return CC_ERR_UNSUPPORTED;
  cudaFuncSetAttribute(k_hv_pull, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  // meeting vertices of degree >= 32 get a warp: find the first such rank
  int32_t x_split = (int32_t)n;
  {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
      int64_t mid = (lo + hi) / 2;
      if (c.cur_graph_row[mid + 1] - c.cur_graph_row[mid] >= 32) hi = mid;
      else lo = mid + 1;
    }
    x_split = (int32_t)lo;
  }
  const int sms = 152;
  for (int64_t top = n - 1; top >= first_rank; top -= B) {
    HvGroup G;
    G.B = (int)std::min<int64_t>(B, top - first_rank + 1);
    G.umax = (int32_t)top;
    for (int b = 0; b < G.B; b++) G.u[b] = (int32_t)(top - b);
    for (int hi = 0; hi < a.n_h; hi++) {
      const int h = a.hs[hi];
      // stamps are cleared with the rows after every group and h: (u, h) is a unique key
      for (int b = 0; b < G.B; b++) G.key[b] = ((unsigned long long)(G.u[b] + 1) << 3) | hi;
      if (cudaMemsetAsync(S.cnt, 0, 2 * kHvLevels * kHvMaxB * sizeof(int), c.stream) != cudaSuccess)
        return CC_ERR_CUDA;
      dim3 g1(std::max<int64_t>(1, std::min<int64_t>(64, (c.cur_graph_row[top + 1] - c.cur_graph_row[top] + 255) / 256)),
              G.B);
      timing_begin(c, "cycle_heavy_levels");
      k_hv_level1<<<g1, 256, 0, c.stream>>>(a, S, G, h);
      c.kernels++;
      for (int hf = 0; hf < 2; hf++)
        if (S.mat[hf] >= 1) {
          k_hv_join<<<sms * 4, 256, 0, c.stream>>>(a, S, G, h, hf, 1);
          c.kernels++;
        }
      for (int j = 1; j < std::max(S.mat[0], S.mat[1]); j++) {
        for (int hf = 0; hf < 2; hf++)
          if (S.mat[hf] >= j + 1) {
            k_hv_push<<<sms * 8, 256, 0, c.stream>>>(a, S, G, h, hf, j);
            c.kernels++;
          }
        for (int hf = 0; hf < 2; hf++)
          if (S.mat[hf] >= j + 1) {
            k_hv_join<<<sms * 4, 256, 0, c.stream>>>(a, S, G, h, hf, j + 1);
            c.kernels++;
          }
      }
      timing_end(c);
      timing_begin(c, "cycle_heavy_pull");
      k_hv_pull<<<sms * 4, kHvThreads, smem, c.stream>>>(a, S, G, h, x_split);
      c.kernels++;
      timing_end(c);
      k_hv_clear<<<sms * 2, 256, 0, c.stream>>>(a, S, G);
      c.kernels++;
      k_hv_finish<<<1, 32, 0, c.stream>>>(a, S, G, hi == a.n_h - 1);
      c.kernels++;
    }
  }
  // leave the level counts at zero as well: the scratch is all zero between launches
  if (cudaMemsetAsync(S.cnt, 0, 2 * kHvLevels * kHvMaxB * sizeof(int), c.stream) != cudaSuccess) return CC_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? CC_OK : CC_ERR_CUDA;
}

}  // namespace cc
