// K5 for unannotated root cycles C_L, L = 4, 5, 6 (k = L): heavy sources in
// groups (level build, pull, closure), the other sources one CTA each (the
// per-CTA push at the end of this file).
//
// The same DB closure as cycle.cu / cycle_heavy.cu, with the table layout
// fixed by the cycle's shape.  For a source u (highest cycle vertex) and a
// meeting vertex x (image of the node opposite a_0), call the colours other
// than chi(u) and chi(x) the free colours (k - 2 of them):
//   * level 1 (paths u -> v): membership only; v contributes its colour;
//   * level 2 (paths u -> v -> w, L = 5, 6): W2[w][c] = number of lower
//     neighbours v of u adjacent to w with chi(v) = c (chi(w), chi(v),
//     chi(u) distinct);
//   * at x, over x's neighbours w below u:
//       A[c]     = number of level-1 neighbours w with chi(w) = c
//       P[{c,d}] = sum of W2[w][d] over level-2 neighbours w with
//                  chi(w) = c, plus the same with c and d exchanged:
//                  the 3-hop half u-v-w-x with colours {chi(v), chi(w)}
//                  = {c, d};
//   * closure over the free colours (Procedure 2, both halves overlapping
//     only in chi(u), chi(x)):
//       C4: 2 A[f0] A[f1]
//       C5: sum_i A[fi] P[{fj, fl}],  {i, j, l} = {0, 1, 2}
//       C6: 2 sum over the three splits {i,j}|{l,m} of P[{fi,fj}] P[{fl,fm}].
// Only one highest node is computed (h = 0) and the total is multiplied by L.
//
// Heavy sources run in groups of 32 (lane b of a warp = source b); A and P
// live in registers.  Two groups are in flight at a time (two scratch
// banks): their level builds run back to back and, for the push-form groups,
// one pull pass serves both.  P entries are exact in 32 bits: a level-2 row
// entry is below 2^16 and x has fewer than 2^16 neighbours (the host checks
// the maximum degree).
#include <algorithm>

#include "cc_kernels.h"

namespace cc {

constexpr int kPcMaxB = 32;  // sources per heavy group (one lane each)
constexpr int kPcThreads = 256;

// colour-tagged adjacency: entry = neighbour | colour << kTagShift (n < 2^29, k <= 8)
constexpr int kTagShift = 29;
constexpr uint32_t kTagMask = (1u << kTagShift) - 1u;

struct PcScratch {
  int64_t n;                   // vertices (bounds-check build)
  u64 *status;                 // status block of the pass (bounds-check build)
  uint16_t *w2;                // [n][32 sources][8 colours] level-2 rows (u16: max degree < 65536)
  unsigned long long *member;  // [n]: bit b level 1 of source b, bit 32+b level 2 (b < 32)
  uint32_t *anym;              // [(n + 31) / 32]: bit w set when w is in some level the pull reads
  int32_t *list;               // [B][n] level-2 vertices (for clearing)
  int *cnt;                    // [B]
  u64 *totals;                 // [B]
};

struct PcGroup {
  int B;
  int32_t u[kPcMaxB];
  int32_t umax;
};

// ------------------------------ level build ------------------------------
// grid.y = source b (of one or two groups); warps walk the lower neighbours v of u_b and their
// neighbours w below u_b, 32 at a time (v's row is rank ordered, so the walk
// stops at the first chunk that reaches u_b).  A level-2 vertex is listed
// once per source, the warp taking its list slots with one atomic.
template <int L>
__global__ void __launch_bounds__(kPcThreads) k_pc_levels(GraphView g, const uint8_t *colors, PcScratch SA,
                                                          PcGroup GA, PcScratch SB, PcGroup GB, u64 *status) {
  constexpr unsigned FULL = 0xffffffffu;
  // rows 0 .. GA.B-1 of the grid serve group A (bank A), the rest group B
  const bool second = (int)blockIdx.y >= GA.B;
  const PcScratch S = second ? SB : SA;
  const PcGroup &G = second ? GB : GA;
  const int b = second ? (int)blockIdx.y - GA.B : (int)blockIdx.y;
  const int32_t u = G.u[b];
  const int cu = colors[u];
  const int64_t n = g.n;
  const int64_t ub = g.row[u];
  const int du = g.lo_cnt[u];
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp0; i < du; i += nwarps) {
    const int32_t v = __ldg(g.col + ub + i);
    if (!cc_in(v, u, status)) continue;
    const int cv = colors[v];
    if (cv == cu) continue;
    if (L <= 5 && lane == 0) {
      atomicOr(S.member + v, 1ull << b);
      atomicOr(S.anym + (v >> 5), 1u << (v & 31));
    }
    if (L == 4) continue;
    const int64_t vb = g.row[v], vend = g.row[v + 1];
    for (int64_t e0 = vb; e0 < vend; e0 += 32) {
      const int64_t e = e0 + lane;
      const int32_t w = e < vend ? __ldg(g.col + e) : INT32_MAX;
      const bool done = __any_sync(FULL, w >= u);
      bool need = false;
      if (w < u && cc_in(w, n, status)) {
        const int cw = colors[w];
        if (cw != cu && cw != cv) {
          // 16-bit counter inside a 32-bit word; counts stay below 2^16 (host check)
          atomicAdd((uint32_t *)(S.w2 + ((int64_t)w * kPcMaxB + b) * 8 + (cv & ~1)), 1u << (16 * (cv & 1)));
          // bits are only set during this kernel, so a stale read can only
          // miss one and cost a redundant atomic; the atomic's old value
          // decides which thread lists w
          if (!((__ldcg(S.member + w) >> (32 + b)) & 1ull)) {
            const unsigned long long old = atomicOr(S.member + w, 1ull << (32 + b));
            need = !((old >> (32 + b)) & 1ull);
            if (need) atomicOr(S.anym + (w >> 5), 1u << (w & 31));
          }
        }
      }
      const unsigned nb = __ballot_sync(FULL, need);
      if (nb) {
        const int leader = __ffs(nb) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(S.cnt + b, __popc(nb));
        base = __shfl_sync(FULL, base, leader);
        if (need && cc_in(base + __popc(nb & lt), n, status)) S.list[(int64_t)b * n + base + __popc(nb & lt)] = w;
      }
      if (done) break;
    }
  }
}

// Pull form of the level build, for groups whose sources reach most of the
// graph (the push form's atomics then collide on the same rows).  First the
// level-1 bits (bit b of member[v] for v in N<(u_b), chi(v) != chi(u_b)),
// then one warp per w below the group's highest source, lane b = source b:
// the warp scans N(w) for level-1 vertices and each lane counts its own
// source's by colour; the row is written where it is non-zero and the upper
// half of member[w] (level-2 bits) is rewritten whole.  Rows whose bit is
// clear are never read, so rows left from the previous group need no
// clearing; the pass as a whole zeroes its scratch once it switches back to
// the push form or ends.
__global__ void k_pc_mark1(GraphView g, const uint8_t *colors, PcScratch S, PcGroup G, bool level1_read,
                           u64 *status) {
  const int b = blockIdx.y;
  const int32_t u = G.u[b];
  const int cu = colors[u];
  const int64_t ub = g.row[u];
  const int du = g.lo_cnt[u];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < du; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = __ldg(g.col + ub + i);
    if (!cc_in(v, u, status)) continue;
    if (colors[v] != cu) {
      atomicOr(S.member + v, 1ull << b);
      if (level1_read) atomicOr(S.anym + (v >> 5), 1u << (v & 31));
    }
  }
}

template <int L>
__device__ __forceinline__ void pc_count(uint32_t (&cnt)[L], int c, uint32_t v) {
  // c is the same in every lane of the warp: the branch does not diverge
  switch (c) {
    case 0: cnt[0] += v; break;
    case 1: cnt[1] += v; break;
    case 2: cnt[2] += v; break;
    case 3: cnt[3] += v; break;
    case 4: if (L > 4) cnt[L > 4 ? 4 : 0] += v; break;
    default: if (L > 5) cnt[L > 5 ? 5 : 0] += v; break;
  }
}

// NG = 1: one group (bank A); NG = 2: groups A and B, each writing its own
// bank, in one pass over the vertices w (the scan of N(w) is shared).
template <int L, int NG>
__global__ void __launch_bounds__(kPcThreads) k_pc_levels_pull(GraphView g, const uint8_t *colors, PcScratch SA,
                                                               PcGroup GA, PcScratch SB, PcGroup GB, u64 *status) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, b = lane;
  bool active[NG];
  int32_t ub[NG];
  int cu[NG];
  // member[v] as two 32-bit halves: [2v] level-1 bits (read here), [2v+1]
  // level-2 bits (written here)
  uint32_t *half[NG];
#pragma unroll
  for (int q = 0; q < NG; q++) {
    const PcGroup &G = q == 0 ? GA : GB;
    active[q] = b < G.B;
    ub[q] = active[q] ? G.u[b] : -1;
    cu[q] = active[q] ? colors[ub[q]] : -1;
    half[q] = reinterpret_cast<uint32_t *>(q == 0 ? SA.member : SB.member);
  }
  const int32_t umax = GA.umax;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t wi = warp0; wi < umax; wi += nwarps) {
    const int32_t w = (int32_t)wi;
    const int cw = colors[w];
    bool act[NG];
    bool any_act = false;
    uint32_t cnt[NG][L];
#pragma unroll
    for (int q = 0; q < NG; q++) {
      act[q] = active[q] && w < ub[q] && cw != cu[q];
      any_act = any_act || act[q];
#pragma unroll
      for (int c = 0; c < L; c++) cnt[q][c] = 0;
    }
    if (__any_sync(FULL, any_act)) {
      const int64_t wb = g.row[w];
      const int deg = (int)(g.row[w + 1] - wb);
      for (int base = 0; base < deg; base += 32) {
        const int j = base + lane;
        int32_t vl = j < deg ? __ldg(g.col + wb + j) : INT32_MAX;
        if (vl < umax && !cc_in(vl, g.n, status)) vl = INT32_MAX;
        const bool past = __any_sync(FULL, vl >= umax);
        uint32_t ml[NG];
        uint32_t mor = 0u;
#pragma unroll
        for (int q = 0; q < NG; q++) {
          ml[q] = vl < umax ? __ldcg(half[q] + 2 * (int64_t)vl) : 0u;
          mor |= ml[q];
        }
        const int cl = mor ? colors[vl] : cw;
        // chi(v) = chi(w): no colourful path u-v-w
        unsigned m = __ballot_sync(FULL, mor != 0u && cl != cw);
        while (m) {
#pragma unroll
          for (int r = 0; r < 4; r++) {
            const int t = m ? __ffs(m) - 1 : 0;
            const bool valid = m != 0u;
            m &= m - 1u;
            const int cc = __shfl_sync(FULL, cl, t);
#pragma unroll
            for (int q = 0; q < NG; q++) {
              const uint32_t mm = __shfl_sync(FULL, ml[q], t);
              if (valid) pc_count<L>(cnt[q], cc, (act[q] && ((mm >> b) & 1u)) ? 1u : 0u);
            }
          }
        }
        if (past) break;
      }
    }
    bool nz_any = false;
#pragma unroll
    for (int q = 0; q < NG; q++) {
      const PcScratch &S = q == 0 ? SA : SB;
      bool nz = false;
#pragma unroll
      for (int c = 0; c < L; c++) nz = nz || cnt[q][c] != 0u;
      if (nz) {
        uint32_t wd[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int c = 0; c < L; c++) wd[c >> 1] |= cnt[q][c] << (16 * (c & 1));
        *(uint4 *)(S.w2 + ((int64_t)w * kPcMaxB + b) * 8) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
      }
      const unsigned bits = __ballot_sync(FULL, nz);
      if (lane == 0) half[q][2 * (int64_t)w + 1] = bits;
      nz_any = nz_any || bits != 0u;
    }
    if (lane == 0 && nz_any) atomicOr(SA.anym + (w >> 5), 1u << (w & 31));
  }
}

// The colour-tagged adjacency of one colouring: tag[e] = col[e] | chi(col[e]) << kTagShift.
__global__ void k_tag_cols(GraphView g, const uint8_t *colors, uint32_t *tag) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < g.nnz; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t w = __ldg(g.col + e);
    tag[e] = (uint32_t)w | ((uint32_t)colors[w] << kTagShift);
  }
}

// Per rank u, the pairs the push form of the level build visits for u as a
// source: v in N<(u), w in N(v) below u.
__global__ void k_push_work(GraphView g, unsigned long long *out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = warp0; u < g.n; u += nwarps) {
    const int64_t ub = g.row[u];
    const int du = g.lo_cnt[u];
    unsigned long long s = 0;
    for (int i = lane; i < du; i += 32) {
      const int32_t v = __ldg(g.col + ub + i);
      const int64_t vb = g.row[v];
      s += (unsigned long long)(lower_bound_i32(g.col, vb, g.row[v + 1], (int32_t)u) - vb);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[u] = s;
  }
}

// ---------------------------------- pull ----------------------------------
__host__ __device__ constexpr int pc_pair(int a, int b) {  // unordered colour pair, a != b
  return a > b ? a * (a - 1) / 2 + b : b * (b - 1) / 2 + a;
}

// Accumulate one level-2 row (w of colour c) into the pair sums:
// P[{c, d}] += W2[w][d] for every colour d != c.  c is a compile-time index.
template <int L, int c>
__device__ __forceinline__ void pc_add_row(uint32_t (&P)[L * (L - 1) / 2], const uint4 &r) {
  const uint32_t wd[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
  for (int d = 0; d < L; d++)
    if (d != c) P[pc_pair(c, d)] += (wd[d >> 1] >> (16 * (d & 1))) & 0xFFFFu;
}

template <int L>
__device__ __forceinline__ void pc_add_row_dyn(uint32_t (&P)[L * (L - 1) / 2], const uint4 &r, int c) {
  // c is the same in every lane of the warp: the branch does not diverge
  switch (c) {
    case 0: pc_add_row<L, 0>(P, r); break;
    case 1: pc_add_row<L, 1>(P, r); break;
    case 2: pc_add_row<L, 2>(P, r); break;
    case 3: pc_add_row<L, 3>(P, r); break;
    case 4: if (L > 4) pc_add_row<L, (L > 4 ? 4 : 0)>(P, r); break;
    default: if (L > 5) pc_add_row<L, (L > 5 ? 5 : 0)>(P, r); break;
  }
}

template <int L>
__device__ __forceinline__ void pc_add_one(uint32_t (&A)[L], int c, uint32_t v) {
#pragma unroll
  for (int i = 0; i < L; i++) A[i] += (c == i) ? v : 0u;
}

// One chunk of 32 neighbours of a meeting vertex x as one lane sees it:
// the neighbour, its colour and its membership word (0 when it cannot
// count: at or above the group's highest source, coloured chi(x), or in no
// source's levels).  The colour comes with the neighbour from the tagged
// adjacency; the membership word is read only where the group's one-bit map
// says the neighbour belongs to some level.
struct PcChunk {
  int32_t w;
  int c;
  unsigned long long m;
};

__device__ __forceinline__ PcChunk pc_load_chunk(const uint32_t *tag, const PcScratch &S, int64_t xb, int deg, int j,
                                                 int cx, int32_t umax) {
  PcChunk k;
  const uint32_t t = j < deg ? __ldg(tag + xb + j) : 0xFFFFFFFFu;
  k.w = j < deg ? (int32_t)(t & kTagMask) : INT32_MAX;
  // a tagged neighbour below the group's highest source is a vertex id
  if (k.w < umax && !cc_in(k.w, S.n, S.status)) k.w = INT32_MAX;
  k.c = k.w < umax ? (int)(t >> kTagShift) : cx;
  const bool any = k.c != cx && ((__ldg(S.anym + (k.w >> 5)) >> (k.w & 31)) & 1u);
  k.m = any ? __ldg(S.member + k.w) : 0ull;
  return k;
}

// Member lanes of a chunk.  C6 reads level-2 bits only (level-1 bits may be
// present from the pull-form build).
template <int L>
__device__ __forceinline__ unsigned pc_members(const PcChunk &k) {
  return __ballot_sync(0xffffffffu, (L >= 6 ? (k.m >> 32) : k.m) != 0ull);
}

// One visited neighbour w (colour c, membership word mm) as lane b sees it.
template <int L>
__device__ __forceinline__ uint4 pc_take(const PcScratch &S, int32_t w, int c, unsigned long long mm, int b,
                                         bool act, int32_t ub, int cu, uint32_t (&A)[L], bool &hit) {
  const bool in = act && w < ub && c != cu;
  if (L <= 5 && in && ((mm >> b) & 1ull)) {
    pc_add_one<L>(A, c, 1u);
    hit = true;
  }
  uint4 r = make_uint4(0, 0, 0, 0);
  if (L >= 5 && in && ((mm >> (32 + b)) & 1ull)) {
    r = __ldg((const uint4 *)(S.w2 + ((int64_t)w * kPcMaxB + b) * 8));
    hit = true;
  }
  return r;
}

// Visit the members of one chunk (mask m): four at a time while at least
// four remain (their level-2 row loads in flight together), then one at a
// time; each lane adds its own source's row.  The visited neighbour's colour
// is the same in all lanes, so a switch on it selects compile-time register
// indices without divergence.
template <int L>
__device__ __forceinline__ void pc_visit_chunk(const PcScratch &S, const PcChunk &k, unsigned m, int b, bool act,
                                               int32_t ub, int cu, uint32_t (&A)[L],
                                               uint32_t (&P)[L * (L - 1) / 2], bool &hit) {
  constexpr unsigned FULL = 0xffffffffu;
  while (__popc(m) >= 4) {
    int32_t ww[4];
    int cc[4];
    unsigned long long mm[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int t = __ffs(m) - 1;
      m &= m - 1u;
      ww[q] = __shfl_sync(FULL, k.w, t);
      cc[q] = __shfl_sync(FULL, k.c, t);
      mm[q] = __shfl_sync(FULL, k.m, t);
    }
    uint4 rr[4];
#pragma unroll
    for (int q = 0; q < 4; q++) rr[q] = pc_take<L>(S, ww[q], cc[q], mm[q], b, act, ub, cu, A, hit);
    if (L >= 5) {
#pragma unroll
      for (int q = 0; q < 4; q++) pc_add_row_dyn<L>(P, rr[q], cc[q]);
    }
  }
  while (m) {
    const int t = __ffs(m) - 1;
    m &= m - 1u;
    const int32_t w = __shfl_sync(FULL, k.w, t);
    const int c = __shfl_sync(FULL, k.c, t);
    const unsigned long long mm = __shfl_sync(FULL, k.m, t);
    const uint4 r = pc_take<L>(S, w, c, mm, b, act, ub, cu, A, hit);
    if (L >= 5) pc_add_row_dyn<L>(P, r, c);
  }
}

// The closure at meeting vertex x for this lane's source, added to tot.  It
// reads the pair sums through shared memory: the free colours depend on
// chi(u), which differs per lane.
template <int L>
__device__ __forceinline__ void pc_close_x(const uint32_t (&A)[L], const uint32_t (&P)[L * (L - 1) / 2], bool on,
                                           int cu, int cx, uint32_t (*sA)[kPcThreads], uint32_t (*sP)[kPcThreads],
                                           int tid, u64 &tot, unsigned &ovf) {
  constexpr int NP = L * (L - 1) / 2;
  if (!on) return;
  // free colours f0 < f1 < ... (all but chi(u) and chi(x))
  uint32_t rest = ((1u << L) - 1u) & ~((1u << cu) | (1u << cx));
  int f[4];
#pragma unroll
  for (int i = 0; i < L - 2; i++) {
    f[i] = __ffs(rest) - 1;
    rest &= rest - 1u;
  }
  if (L <= 5) {
#pragma unroll
    for (int c = 0; c < L; c++) sA[c][tid] = A[c];
  }
  if (L >= 5) {
#pragma unroll
    for (int j = 0; j < NP; j++) sP[j][tid] = P[j];
  }
  if (L == 4) {
    tot = add_ck(tot, mul_ck(2ull, mul_ck(sA[f[0]][tid], sA[f[1]][tid], ovf), ovf), ovf);
  } else if (L == 5) {
    u64 t = mul_ck(sA[f[0]][tid], sP[pc_pair(f[1], f[2])][tid], ovf);
    t = add_ck(t, mul_ck(sA[f[1]][tid], sP[pc_pair(f[0], f[2])][tid], ovf), ovf);
    t = add_ck(t, mul_ck(sA[f[2]][tid], sP[pc_pair(f[0], f[1])][tid], ovf), ovf);
    tot = add_ck(tot, t, ovf);
  } else {
    u64 t = (u64)sP[pc_pair(f[0], f[1])][tid] * sP[pc_pair(f[2], f[3])][tid];
    t = add_ck(t, (u64)sP[pc_pair(f[0], f[2])][tid] * sP[pc_pair(f[1], f[3])][tid], ovf);
    t = add_ck(t, (u64)sP[pc_pair(f[0], f[3])][tid] * sP[pc_pair(f[1], f[2])][tid], ovf);
    tot = add_ck(tot, mul_ck(2ull, t, ovf), ovf);
  }
}

// All chunks of one meeting vertex (the first one already loaded) and the
// closure at it, added to tot.
template <int L>
__device__ __forceinline__ void pc_meet(const uint32_t *tag, const PcScratch &S, int32_t x,
                                        int cx, int64_t xb, int deg, PcChunk k, int lane, bool active, int32_t ub,
                                        int cu, int32_t umax, uint32_t (*sA)[kPcThreads],
                                        uint32_t (*sP)[kPcThreads], int tid, u64 &tot, unsigned &ovf) {
  constexpr int NP = L * (L - 1) / 2;
  constexpr unsigned FULL = 0xffffffffu;
  const bool act = active && x < ub && cx != cu;
  // the row is rank ordered: past the highest source, nothing further counts
  bool past = __any_sync(FULL, k.w >= umax);
  unsigned m = pc_members<L>(k);
  if (!m && (past || deg <= 32)) return;  // x meets no member
  if (!__any_sync(FULL, act)) return;
  uint32_t A[L], P[NP];
#pragma unroll
  for (int c = 0; c < L; c++) A[c] = 0;
#pragma unroll
  for (int j = 0; j < NP; j++) P[j] = 0;
  bool hit = false;
  for (int base = 0;;) {
    pc_visit_chunk<L>(S, k, m, lane, act, ub, cu, A, P, hit);
    base += 32;
    if (past || base >= deg) break;
    k = pc_load_chunk(tag, S, xb, deg, base + lane, cx, umax);
    past = __any_sync(FULL, k.w >= umax);
    m = pc_members<L>(k);
  }
  pc_close_x<L>(A, P, act && hit, cu, cx, sA, sP, tid, tot, ovf);
}

// One warp per meeting vertex x below the group's highest source, lane b =
// source b.
template <int L>
__global__ void __launch_bounds__(kPcThreads, 4) k_pc_pull(GraphView g, const uint32_t *tag, PcScratch S, PcGroup G,
                                                        const uint8_t *colors, u64 *status) {
  constexpr int NP = L * (L - 1) / 2;
  __shared__ uint32_t sP[L >= 5 ? NP : 1][kPcThreads];
  __shared__ uint32_t sA[L <= 5 ? L : 1][kPcThreads];
  const int tid = threadIdx.x, lane = tid & 31, b = lane;
  const bool active = b < G.B;
  const int32_t ub = active ? G.u[b] : -1;
  const int cu = active ? colors[ub] : -1;
  const int32_t umax = G.umax;
  u64 tot = 0;
  unsigned ovf = 0;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t xi = warp0; xi < umax; xi += nwarps) {
    const int32_t x = (int32_t)xi;
    const int cx = colors[x];
    const int64_t xb = g.row[x];
    const int deg = (int)(g.row[x + 1] - xb);
    const PcChunk k = pc_load_chunk(tag, S, xb, deg, lane, cx, umax);
    pc_meet<L>(tag, S, x, cx, xb, deg, k, lane, active, ub, cu, umax, sA, sP, tid, tot, ovf);
  }
  if (active && tot) atomic_add_ck(S.totals + b, tot, ovf);
  flag_overflow(status, ovf);
}

// Two groups in one pass over the meeting vertices (groups A and B, A the
// higher, each with its own scratch bank and a member map shared by both):
// the scan of x -- row bounds, the first chunk of tagged neighbours, the
// member map -- is paid once for 64 sources; each group is then visited and
// closed as in k_pc_pull (lane b = source b of A, then of B).
template <int L>
__global__ void __launch_bounds__(kPcThreads, 4) k_pc_pull2(GraphView g, const uint32_t *tag, PcScratch SA, PcGroup GA,
                                                         PcScratch SB, PcGroup GB, const uint8_t *colors,
                                                         u64 *status) {
  constexpr int NP = L * (L - 1) / 2;
  __shared__ uint32_t sP[L >= 5 ? NP : 1][kPcThreads];
  __shared__ uint32_t sA[L <= 5 ? L : 1][kPcThreads];
  const int tid = threadIdx.x, lane = tid & 31, b = lane;
  const bool actA = b < GA.B, actB = b < GB.B;
  const int32_t ubA = actA ? GA.u[b] : -1, ubB = actB ? GB.u[b] : -1;
  const int cuA = actA ? colors[ubA] : -1, cuB = actB ? colors[ubB] : -1;
  const int32_t umax = GA.umax;
  u64 totA = 0, totB = 0;
  unsigned ovf = 0;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t xi = warp0; xi < umax; xi += nwarps) {
    const int32_t x = (int32_t)xi;
    const int cx = colors[x];
    const int64_t xb = g.row[x];
    const int deg = (int)(g.row[x + 1] - xb);
    const uint32_t t = lane < deg ? __ldg(tag + xb + lane) : 0xFFFFFFFFu;
    PcChunk kA;
    kA.w = lane < deg ? (int32_t)(t & kTagMask) : INT32_MAX;
    if (kA.w < umax && !cc_in(kA.w, g.n, status)) kA.w = INT32_MAX;
    kA.c = kA.w < umax ? (int)(t >> kTagShift) : cx;
    const bool any = kA.c != cx && ((__ldg(SA.anym + (kA.w >> 5)) >> (kA.w & 31)) & 1u);
    kA.m = any ? __ldg(SA.member + kA.w) : 0ull;
    PcChunk kB = kA;
    kB.m = any ? __ldg(SB.member + kA.w) : 0ull;
    pc_meet<L>(tag, SA, x, cx, xb, deg, kA, lane, actA, ubA, cuA, umax, sA, sP, tid, totA, ovf);
    pc_meet<L>(tag, SB, x, cx, xb, deg, kB, lane, actB, ubB, cuB, umax, sA, sP, tid, totB, ovf);
  }
  if (actA && totA) atomic_add_ck(SA.totals + b, totA, ovf);
  if (actB && totB) atomic_add_ck(SB.totals + b, totB, ovf);
  flag_overflow(status, ovf);
}

// --------------------------- clear and finish ---------------------------
// grid.y = source b: zero its level-1 membership words and, for its listed
// level-2 vertices, the membership word, the row and the list entry.
template <int L>
__global__ void k_pc_clear(GraphView g, PcScratch SA, PcGroup GA, PcScratch SB, PcGroup GB, u64 *status) {
  // rows 0 .. GA.B-1 of the grid serve group A (bank A), the rest group B
  const bool second = (int)blockIdx.y >= GA.B;
  const PcScratch S = second ? SB : SA;
  const PcGroup &G = second ? GB : GA;
  const int b = second ? (int)blockIdx.y - GA.B : (int)blockIdx.y;
  const int64_t n = g.n;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nt = (int64_t)gridDim.x * blockDim.x;
  const int32_t u = G.u[b];
  const int64_t ub = g.row[u];
  const int du = g.lo_cnt[u];
  for (int64_t i = t0; i < du; i += nt) {
    const int32_t v = __ldg(g.col + ub + i);
    if (cc_in(v, n, status)) S.member[v] = 0;
  }
  if (L >= 5) {
    const int cnt = S.cnt[b];
    for (int64_t i = t0; i < cnt; i += nt) {
      const int32_t w = S.list[(int64_t)b * n + i];
      S.list[(int64_t)b * n + i] = 0;
      if (!cc_in(w, n, status)) continue;
      S.member[w] = 0;
      *(uint4 *)(S.w2 + ((int64_t)w * kPcMaxB + b) * 8) = make_uint4(0, 0, 0, 0);
    }
  }
}

// One lane per source (one warp per group): the totals (times the rotation multiplier)
// into the per-vertex split and the count; totals and list counts back to 0.
__global__ void k_pc_finish(PcScratch SA, PcGroup GA, PcScratch SB, PcGroup GB, int multiplier, u64 *per_vertex,
                            u64 *status) {
  // warp 0: group A, warp 1 (when launched): group B
  const bool second = threadIdx.x >= 32;
  const PcScratch S = second ? SB : SA;
  const PcGroup &G = second ? GB : GA;
  const int b = threadIdx.x & 31;
  unsigned ovf = 0;
  u64 t = 0;
  if (b < G.B) {
    t = mul_ck(S.totals[b], (u64)multiplier, ovf);
    S.totals[b] = 0;
    S.cnt[b] = 0;
    if (per_vertex) per_vertex[G.u[b]] = t;
  }
  t = warp_sum_ck(t, ovf);
  if (b == 0 && t) atomic_add_ck(status + ST_COUNT, t, ovf);
  flag_overflow(status, ovf);
}

// ------------------- light and medium sources: one CTA each -------------------
// Sources of degree below the heavy threshold have small reach sets, so the
// last hop is pushed: every level-2 vertex w adds its row into the level-3
// row of each lower neighbour x (u32, indexed by the unordered pair of free
// colours), and the closure runs over the touched meeting vertices only.
// u32 is exact here: a level-3 entry counts paths u-v-w-x and is at most
// deg(x) * deg(u), which the host checks stays below 2^32.
//
// The rows of one source are compact: a vertex reached at level 2 (3) gets
// the next local index, and its row lives at that index, so the rows a source
// touches are contiguous and stay in cache.  Each level is walked once: a
// thread reaching v swaps id[v] from 0 to -1; the winner takes the next index,
// lists v and publishes id[v] = index + 1, every other thread reads the index
// from the swap's old value (or, in the short window before the winner
// publishes, waits for it, with an iteration limit that reports
// CC_ERR_TIMEOUT), and then adds into v's row.
#ifndef CC_PL_THREADS
#define CC_PL_THREADS 256
#endif
#ifndef CC_PL_SLOTS_PER_SM
#define CC_PL_SLOTS_PER_SM (1024 / CC_PL_THREADS)
#endif
constexpr int kPlThreads = CC_PL_THREADS;          // threads per source (one CTA)
constexpr int kPlSlotsPerSM = CC_PL_SLOTS_PER_SM;  // resident CTAs per SM, one scratch slot each

__device__ __forceinline__ int pair_idx(int a, int b) {
  int hi = a > b ? a : b, lo = a > b ? b : a;
  return hi * (hi - 1) / 2 + lo;
}

#ifdef CC_TEST_WAIT_EXPIRES
// Test build (libcc_waittest.so) only: every thread that finds v already
// claimed enters the wait as if the claimant had not published yet, and the
// wait gives up at once, so the report of a wait that ran out reaches the
// caller deterministically.  No access changes: the contribution is skipped.
constexpr int kPlSpinLimit = 0;
#else
constexpr int kPlSpinLimit = 1 << 22;
#endif

// Local index of v at one level: claimed (and listed) by the first thread to
// reach it, read by the others; -1 when the wait for the claimant gave up.
__device__ __forceinline__ int pl_index(int32_t *id, int32_t v, int32_t *list, int *s_n, unsigned &tmo) {
  int old = atomicCAS(id + v, 0, -1);
  if (old == 0) {
    const int i = atomicAdd(s_n, 1);
    list[i] = v;
    atomicExch(id + v, i + 1);
    return i;
  }
#ifdef CC_TEST_WAIT_EXPIRES
  old = -1;
#endif
  for (int spins = 0; old < 0; spins++) {
    if (spins == kPlSpinLimit) {
      tmo = 1u;
      return -1;
    }
    old = *(volatile int32_t *)(id + v);
  }
  return old - 1;
}

template <int L>
__global__ void __launch_bounds__(kPlThreads) k_pc_light(GraphView g, const uint8_t *colors, PlScratch S,
                                                         int32_t end_rank, int *work, int multiplier,
                                                         u64 *per_vertex, u64 *status, int k) {
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ int s_u, s_n2, s_n3;
  __shared__ unsigned long long s_tot;
  __shared__ unsigned s_ovf;
  char *slot = S.base + (size_t)blockIdx.x * S.slot_bytes;
  uint32_t *W2 = (uint32_t *)(slot + S.o_w2);   // [local][8] level-2 rows by colour of v
  uint32_t *W3 = (uint32_t *)(slot + S.o_w3);   // [local][16] level-3 rows by colour pair
  int32_t *id2 = (int32_t *)(slot + S.o_mark);  // [n] local index + 1 at level 2 (0 none, -1 claimed)
  int32_t *id3 = (int32_t *)(slot + S.o_id3);   // [n] the same at level 3
  int32_t *L2 = (int32_t *)(slot + S.o_l2);     // local index -> vertex
  int32_t *L3 = (int32_t *)(slot + S.o_l3);
  const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
  constexpr int NW = kPlThreads / 32;
  while (true) {
    if (tid == 0) {
      s_u = end_rank - 1 - atomicAdd(work, 1);
      s_n2 = 0;
      s_n3 = 0;
      s_tot = 0;
      s_ovf = 0;
    }
    __syncthreads();
    const int32_t u = s_u;
    if (u < 0) break;
    const int cu = colors[u];
    const int64_t ub = g.row[u];
    const int du = g.lo_cnt[u];
    unsigned ovf = 0, tmo = 0;
    if (du >= 2) {
      // level 2: pairs (v, w), v in N<(u), w in N(v) below u: chi(v) counted
      // into w's row.  v's row is rank ordered: it is walked to the first
      // chunk that reaches u.
      for (int i = wib; i < du; i += NW) {
        const int32_t v = __ldg(g.col + ub + i);
        if (!cc_in(v, u, status)) continue;
        const int cv = colors[v];
        if (cv == cu) continue;
        const int64_t vb = g.row[v], vend = g.row[v + 1];
        for (int64_t e0 = vb; e0 < vend; e0 += 32) {
          const int64_t e = e0 + lane;
          const int32_t w = e < vend ? __ldg(g.col + e) : INT32_MAX;
          const bool done = __any_sync(FULL, w >= u);
          if (w < u && cc_in(w, g.n, status)) {
            const int cw = colors[w];
            if (cw != cu && cw != cv) {
              const int iw = pl_index(id2, w, L2, &s_n2, tmo);
              if (iw >= 0 && cc_in(iw, g.n, status)) atomicAdd(W2 + (int64_t)iw * 8 + cv, 1u);
            }
          }
          if (done) break;
        }
      }
      __syncthreads();
      const int n2 = s_n2;
      if (L >= 5) {
        // level 3: pairs (w, x), w a level-2 vertex, x in N(w) below u: w's
        // row added into x's pair row
        for (int i = wib; i < n2; i += NW) {
          const int32_t w = L2[i];
          if (!cc_in(w, g.n, status)) continue;
          const int cw = colors[w];
          const uint4 r0 = *(const uint4 *)(W2 + (int64_t)i * 8);
          const uint4 r1 = *(const uint4 *)(W2 + (int64_t)i * 8 + 4);
          const uint32_t row[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
          const int64_t wb = g.row[w], wend = g.row[w + 1];
          for (int64_t e0 = wb; e0 < wend; e0 += 32) {
            const int64_t e = e0 + lane;
            const int32_t x = e < wend ? __ldg(g.col + e) : INT32_MAX;
            const bool done = __any_sync(FULL, x >= u);
            if (x < u && cc_in(x, g.n, status)) {
              const int cx = colors[x];
              if (cx != cu && cx != cw) {
                bool any = false;
#pragma unroll
                for (int c = 0; c < 8; c++) any = any || (row[c] != 0u && c != cx);
                if (any) {
                  const int ix = pl_index(id3, x, L3, &s_n3, tmo);
                  if (ix >= 0 && cc_in(ix, g.n, status)) {
#pragma unroll
                    for (int c = 0; c < 8; c++) {
                      const uint32_t t = row[c];
                      if (t && c != cx) atomicAdd(W3 + (int64_t)ix * 16 + pair_idx(cw, c), t);
                    }
                  }
                }
              }
            }
            if (done) break;
          }
        }
        __syncthreads();
      }
      // closure at the meeting vertices (level 3 for L >= 5, level 2 for L = 4)
      const int nx = L >= 5 ? s_n3 : n2;
      u64 mine = 0;
      for (int i = tid; i < nx; i += kPlThreads) {
        const int32_t x = L >= 5 ? L3[i] : L2[i];
        if (!cc_in(x, g.n, status)) continue;
        const int cx = colors[x];
        const uint32_t fm = ((1u << k) - 1u) & ~((1u << cu) | (1u << cx));
        int f[4];
        uint32_t rest = fm;
#pragma unroll
        for (int j = 0; j < L - 2; j++) {
          f[j] = __ffs(rest) - 1;
          rest &= rest - 1;
        }
        if (L == 4) {
          const uint32_t *w2 = W2 + (int64_t)i * 8;
          const u64 a0 = w2[f[0]], a1 = w2[f[1]];
          mine = add_ck(mine, mul_ck(2ull, mul_ck(a0, a1, ovf), ovf), ovf);
        } else if (L == 5) {
          const uint32_t *w3 = W3 + (int64_t)i * 16;
          const int ix = id2[x];  // x's level-2 row (paths u-v-x), if x was reached at level 2
          if (ix > 0 && cc_in(ix - 1, g.n, status)) {
            const uint32_t *w2 = W2 + (int64_t)(ix - 1) * 8;
            u64 t = mul_ck((u64)w2[f[0]], (u64)w3[pair_idx(f[1], f[2])], ovf);
            t = add_ck(t, mul_ck((u64)w2[f[1]], (u64)w3[pair_idx(f[0], f[2])], ovf), ovf);
            t = add_ck(t, mul_ck((u64)w2[f[2]], (u64)w3[pair_idx(f[0], f[1])], ovf), ovf);
            mine = add_ck(mine, t, ovf);
          }
        } else {
          const uint32_t *w3 = W3 + (int64_t)i * 16;
          u64 t = mul_ck((u64)w3[pair_idx(f[0], f[1])], (u64)w3[pair_idx(f[2], f[3])], ovf);
          t = add_ck(t, mul_ck((u64)w3[pair_idx(f[0], f[2])], (u64)w3[pair_idx(f[1], f[3])], ovf), ovf);
          t = add_ck(t, mul_ck((u64)w3[pair_idx(f[0], f[3])], (u64)w3[pair_idx(f[1], f[2])], ovf), ovf);
          mine = add_ck(mine, mul_ck(2ull, t, ovf), ovf);
        }
      }
      mine = warp_sum_ck(mine, ovf);
      if (lane == 0 && mine) {
        unsigned long long old = atomicAdd(&s_tot, mine);
        if (old + mine < old) ovf = 1;
      }
      __syncthreads();
      // everything back to zero: rows by local index, ids through the lists
      if (L >= 5) {
        for (int i = tid; i < s_n3; i += kPlThreads) {
          if (cc_in(L3[i], g.n, status)) id3[L3[i]] = 0;
          L3[i] = 0;
          uint4 *z = (uint4 *)(W3 + (int64_t)i * 16);
          z[0] = z[1] = z[2] = z[3] = make_uint4(0, 0, 0, 0);
        }
      }
      for (int i = tid; i < n2; i += kPlThreads) {
        if (cc_in(L2[i], g.n, status)) id2[L2[i]] = 0;
        L2[i] = 0;
        uint4 *z = (uint4 *)(W2 + (int64_t)i * 8);
        z[0] = z[1] = make_uint4(0, 0, 0, 0);
      }
    }
    if (ovf) atomicOr(&s_ovf, 1u);
    if (tmo) atomicOr(status + ST_TIMEOUT, 1ull);
    __syncthreads();
    if (tid == 0) {
      unsigned o = s_ovf;
      u64 t = mul_ck(s_tot, (u64)multiplier, o);
      if (per_vertex) per_vertex[u] = t;
      if (t) atomic_add_ck(status + ST_COUNT, t, o);
      if (o) atomicOr(status + ST_OVERFLOW, 1ull);
    }
    __syncthreads();
  }
}

// Launch the per-CTA push kernel on caller-provided scratch (no allocation
// here): `slots` CTAs, scratch slots laid out from S.base, *work zeroed by
// the caller, sources 0 .. end_rank-1 (the highest first).
int launch_pc_light_raw(cudaStream_t stream, int L, const GraphView &g, const uint8_t *colors, const PlScratch &S,
                        int slots, int32_t end_rank, int *work, u64 *status, int k) {
  if (L == 4)
    k_pc_light<4><<<slots, kPlThreads, 0, stream>>>(g, colors, S, end_rank, work, L, nullptr, status, k);
  else if (L == 5)
    k_pc_light<5><<<slots, kPlThreads, 0, stream>>>(g, colors, S, end_rank, work, L, nullptr, status, k);
  else if (L == 6)
    k_pc_light<6><<<slots, kPlThreads, 0, stream>>>(g, colors, S, end_rank, work, L, nullptr, status, k);
  else
    return CC_ERR_INVALID_ARG;
  return cudaGetLastError() == cudaSuccess ? CC_OK : CC_ERR_CUDA;
}

int run_plain_light(Ctx &c, const CycleArgs &a, int32_t end_rank) {
  if (end_rank <= 0) return CC_OK;
  const int64_t n = a.g.n;
  PlScratch S;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  S.o_w2 = take((size_t)n * 32);
  S.o_w3 = a.L >= 5 ? take((size_t)n * 64) : 0;
  S.o_mark = take((size_t)n * 4);
  S.o_id3 = a.L >= 5 ? take((size_t)n * 4) : 0;
  S.o_l2 = take((size_t)n * 4);
  S.o_l3 = a.L >= 5 ? take((size_t)n * 4) : 0;
  S.slot_bytes = off;
  // one slot per resident CTA (up to four per SM); without a budget, slots
  // take at most a quarter of the free device memory and 64 GiB.  A scratch
  // already large enough for more slots is used whole, and under stream
  // capture only the scratch at hand is used (no allocation).
  constexpr int kMaxSlots = 152 * kPlSlotsPerSM;
  const size_t have = c.scratch_bytes > 256 ? (c.scratch_bytes - 256) / std::max<size_t>(1, S.slot_bytes) : 0;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(c.stream, &cs) != cudaSuccess) return CC_ERR_CUDA;
  int slots;
  if (cs != cudaStreamCaptureStatusNone && have >= 1) {
    slots = (int)std::min<size_t>(kMaxSlots, have);
  } else {
    size_t budget;
    if (c.budget) {
      budget = c.budget > c.in_use ? (c.budget - c.in_use) / 2 : 0;
    } else {
      size_t fr = 0, tot = 0;
      if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return CC_ERR_CUDA;
      budget = std::min<size_t>(fr / 4, (size_t)64 << 30);
    }
    slots = (int)std::max<size_t>(std::min<size_t>(kMaxSlots, budget / std::max<size_t>(1, S.slot_bytes)),
                                  std::min<size_t>(kMaxSlots, have));
  }
  if (slots < 1) return CC_ERR_OOM;
  size_t need = (size_t)slots * S.slot_bytes + 256;
  int rc = ensure_scratch(c, need);
  if (rc != CC_OK) return rc;
  S.base = (char *)c.scratch;
  int *work = (int *)((char *)c.scratch + (size_t)slots * S.slot_bytes);
  if (c.scratch_dirty) {
    if (cudaMemsetAsync(c.scratch, 0, c.scratch_bytes, c.stream) != cudaSuccess) return CC_ERR_CUDA;
    c.scratch_dirty = false;
  }
  if (cudaMemsetAsync(work, 0, sizeof(int), c.stream) != cudaSuccess) return CC_ERR_CUDA;
  timing_begin(c, "cycle_plain_light");
  if (a.L == 4)
    k_pc_light<4><<<slots, kPlThreads, 0, c.stream>>>(a.g, a.colors, S, end_rank, work, a.multiplier,
                                                       a.per_vertex, a.status, a.k);
  else if (a.L == 5)
    k_pc_light<5><<<slots, kPlThreads, 0, c.stream>>>(a.g, a.colors, S, end_rank, work, a.multiplier,
                                                       a.per_vertex, a.status, a.k);
  else
    k_pc_light<6><<<slots, kPlThreads, 0, c.stream>>>(a.g, a.colors, S, end_rank, work, a.multiplier,
                                                       a.per_vertex, a.status, a.k);
  c.kernels++;
  timing_end(c);
  // the queue counter returns to zero too: the whole scratch is zero between launches
  if (cudaMemsetAsync(work, 0, sizeof(int), c.stream) != cudaSuccess) return CC_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? CC_OK : CC_ERR_CUDA;
}

// Push-form work per source rank, computed once per graph (host copy).
// Under stream capture it is not computed: the push form is then used.
static int push_work(Ctx &c, const GraphView &g, const int64_t **out) {
  *out = nullptr;
  DevGraph *dg = c.cur_graph;
  if (!dg) return CC_OK;
  if (dg->h_push_work.empty()) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c.stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return CC_OK;
    const size_t bytes = (size_t)g.n * 8;
    u64 *d = (u64 *)dev_alloc(c, bytes);
    if (!d) return CC_ERR_OOM;
    k_push_work<<<152 * 8, 256, 0, c.stream>>>(g, d);
    c.kernels++;
    std::vector<int64_t> h((size_t)g.n);
    const bool ok = cudaMemcpyAsync(h.data(), d, bytes, cudaMemcpyDeviceToHost, c.stream) == cudaSuccess &&
                    cudaStreamSynchronize(c.stream) == cudaSuccess;
    dev_free(c, d, bytes);
    if (!ok) return CC_ERR_CUDA;
    dg->h_push_work.swap(h);
  }
  *out = dg->h_push_work.data();
  return CC_OK;
}

// A group takes the pull-form level build while its push work exceeds this
// many times the edges of the rows below its highest source (the pull form
// scans those rows once, without atomics).
constexpr double kPullLevelsRatio = 0.5;

template <int L>
static int run_plain_L(Ctx &c, const CycleArgs &a, int32_t first_rank, const PcScratch *SB, const uint32_t *tag) {
  const int64_t n = a.g.n;
  const int sms = 152;
  const PcScratch &S0 = SB[0], &S1 = SB[1];
  const int64_t *pw = nullptr;
  if (L >= 5) {
    int rc = push_work(c, a.g, &pw);
    if (rc != CC_OK) return rc;
  }
  // groups of the pull-form level build leave their banks to be zeroed
  bool pulled_b1 = false;  // bank 1 served a pull-form group
  auto zero_levels = [&]() {
    for (int q = 0; q < (pulled_b1 ? 2 : 1); q++) {
      const PcScratch &S = q == 0 ? S0 : S1;
      if (cudaMemsetAsync(S.member, 0, (size_t)n * 8, c.stream) != cudaSuccess ||
          cudaMemsetAsync(S.w2, 0, (size_t)kPcMaxB * n * 16, c.stream) != cudaSuccess)
        return false;
    }
    return true;
  };
  auto group_at = [&](int64_t top) {
    PcGroup G;
    G.B = (int)std::min<int64_t>(kPcMaxB, top - first_rank + 1);
    G.umax = (int32_t)top;
    for (int b = 0; b < G.B; b++) G.u[b] = (int32_t)(top - b);
    return G;
  };
  PcGroup none;
  none.B = 0;
  none.umax = 0;
  // push-form level build of one group (G2.B = 0) or two (banks 0 and 1);
  // grid rows are sources, the highest source's degree sizes the grid
  auto push_levels = [&](const PcGroup &G, const PcGroup &G2) {
    const int64_t du = c.cur_graph_row[G.umax + 1] - c.cur_graph_row[G.umax];
    dim3 gl((unsigned)std::max<int64_t>(1, std::min<int64_t>(sms * 2, (du * 32 + kPcThreads - 1) / kPcThreads)),
            G.B + G2.B);
    k_pc_levels<L><<<gl, kPcThreads, 0, c.stream>>>(a.g, a.colors, S0, G, S1, G2, a.status);
    c.kernels++;
  };
  // scratch of one group (bank 0) or two back to zero; totals into the count
  auto close_groups = [&](const PcGroup &G, const PcGroup &G2) {
    k_pc_clear<L><<<dim3(std::max(1, sms / 8), G.B + G2.B), 256, 0, c.stream>>>(a.g, S0, G, S1, G2, a.status);
    c.kernels++;
    k_pc_finish<<<1, G2.B ? 64 : 32, 0, c.stream>>>(S0, G, S1, G2, a.multiplier, a.per_vertex, a.status);
    c.kernels++;
  };
  const size_t anym_bytes = (size_t)((n + 31) / 32) * 4;
  k_tag_cols<<<sms * 8, 256, 0, c.stream>>>(a.g, a.colors, (uint32_t *)tag);
  c.kernels++;
  bool pulled = false, pushed = false;
  for (int64_t top = n - 1; top >= first_rank;) {
    const PcGroup G = group_at(top);
    // the pull form serves a prefix of the groups (the highest sources)
    bool use_pull = false;
    if (pw && !pushed) {
      double work = 0;
      for (int b = 0; b < G.B; b++) work += (double)pw[G.u[b]];
      use_pull = work > kPullLevelsRatio * (double)c.cur_graph_row[top];
    }
    if (!use_pull && pulled && !pushed && !zero_levels()) return CC_ERR_CUDA;
    // the one-bit member map is rebuilt for every pass
    if (cudaMemsetAsync(S0.anym, 0, anym_bytes, c.stream) != cudaSuccess) return CC_ERR_CUDA;
    if (use_pull) {
      // pull form, two groups per pass when the next one qualifies too
      bool two = false;
      PcGroup G2 = G;
      if (top - kPcMaxB >= first_rank) {
        G2 = group_at(top - kPcMaxB);
        double work = 0;
        for (int b = 0; b < G2.B; b++) work += (double)pw[G2.u[b]];
        two = work > kPullLevelsRatio * (double)c.cur_graph_row[G2.umax];
      }
      timing_begin(c, "cycle_plain_levels_pull");
      for (int q = 0; q < (two ? 2 : 1); q++) {
        const PcGroup &Gq = q == 0 ? G : G2;
        const int64_t du = c.cur_graph_row[Gq.umax + 1] - c.cur_graph_row[Gq.umax];
        dim3 gm((unsigned)std::max<int64_t>(1, std::min<int64_t>(sms, (du + kPcThreads - 1) / kPcThreads)), Gq.B);
        k_pc_mark1<<<gm, kPcThreads, 0, c.stream>>>(a.g, a.colors, q == 0 ? S0 : S1, Gq, L <= 5, a.status);
        c.kernels++;
      }
      if (two)
        k_pc_levels_pull<L, 2><<<sms * 4, kPcThreads, 0, c.stream>>>(a.g, a.colors, S0, G, S1, G2, a.status);
      else
        k_pc_levels_pull<L, 1><<<sms * 4, kPcThreads, 0, c.stream>>>(a.g, a.colors, S0, G, S0, G, a.status);
      c.kernels++;
      timing_end(c);
      // dense members: each group pulled on its own (the shared scan is a
      // small part of these groups' pull)
      timing_begin(c, "cycle_plain_pull");
      k_pc_pull<L><<<sms * 4, kPcThreads, 0, c.stream>>>(a.g, tag, S0, G, a.colors, a.status);
      c.kernels++;
      if (two) {
        k_pc_pull<L><<<sms * 4, kPcThreads, 0, c.stream>>>(a.g, tag, S1, G2, a.colors, a.status);
        c.kernels++;
      }
      timing_end(c);
      close_groups(G, two ? G2 : none);
      pulled = true;
      pulled_b1 = pulled_b1 || two;
      top -= two ? 2 * kPcMaxB : kPcMaxB;
      continue;
    }
    // push form: two groups per pass when two remain
    pushed = true;
    const bool two = top - kPcMaxB >= first_rank;
    const PcGroup G2 = two ? group_at(top - kPcMaxB) : G;
    timing_begin(c, "cycle_plain_levels");
    push_levels(G, two ? G2 : none);
    timing_end(c);
    timing_begin(c, "cycle_plain_pull");
    if (two)
      k_pc_pull2<L><<<sms * 4, kPcThreads, 0, c.stream>>>(a.g, tag, S0, G, S1, G2, a.colors, a.status);
    else
      k_pc_pull<L><<<sms * 4, kPcThreads, 0, c.stream>>>(a.g, tag, S0, G, a.colors, a.status);
    c.kernels++;
    timing_end(c);
    close_groups(G, two ? G2 : none);
    top -= two ? 2 * kPcMaxB : kPcMaxB;
  }
  // the scratch is all zero between launches
  if (pulled && !pushed && !zero_levels()) return CC_ERR_CUDA;
  if (cudaMemsetAsync(S0.anym, 0, anym_bytes, c.stream) != cudaSuccess) return CC_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? CC_OK : CC_ERR_CUDA;
}

bool plain_cycle_eligible(const CycleArgs &a) {
  if (a.L < 4 || a.L > 6 || a.k != a.L || a.n_h != 1) return false;
  for (int i = 0; i < a.L; i++)
    if (a.N[i].p || a.Efw[i].p || a.Ebw[i].p) return false;
  return true;
}

int run_plain_heavy(Ctx &c, const CycleArgs &a, int32_t first_rank) {
  const int64_t n = a.g.n;
  if (first_rank >= n) return CC_OK;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  const bool lv2 = a.L >= 5;
  // two banks of per-group scratch (two groups pulled together) and one
  // member map shared by them
  size_t o_w2[2], o_mem[2], o_list[2], o_cnt[2], o_tot[2];
  for (int k = 0; k < 2; k++) {
    o_w2[k] = lv2 ? take((size_t)kPcMaxB * n * 8 * 2) : 0;
    o_mem[k] = take((size_t)n * 8);
    o_list[k] = lv2 ? take((size_t)kPcMaxB * n * 4) : 0;
    o_cnt[k] = take(kPcMaxB * 4);
    o_tot[k] = take(kPcMaxB * 8);
  }
  size_t o_anym = take((size_t)((n + 31) / 32) * 4);
  size_t need = off;
  int rc0 = ensure_hv_scratch(c, need);
  if (rc0 != CC_OK) return rc0;
  char *base = (char *)c.hv_scratch;
  PcScratch S[2];
  for (int k = 0; k < 2; k++) {
    S[k].n = n;
    S[k].status = a.status;
    S[k].w2 = (uint16_t *)(base + o_w2[k]);
    S[k].member = (unsigned long long *)(base + o_mem[k]);
    S[k].list = (int32_t *)(base + o_list[k]);
    S[k].cnt = (int *)(base + o_cnt[k]);
    S[k].totals = (u64 *)(base + o_tot[k]);
    S[k].anym = (uint32_t *)(base + o_anym);
  }
  // the tagged adjacency is rewritten every pass: it lives outside the
  // heavy scratch, whose contents are zero between launches
  if ((rc0 = ensure_tag_scratch(c, (size_t)std::max<int64_t>(a.g.nnz, 1) * 4)) != CC_OK) return rc0;
  const uint32_t *tag = (const uint32_t *)c.tag_scratch;
  if (a.L == 4) return run_plain_L<4>(c, a, first_rank, S, tag);
  if (a.L == 5) return run_plain_L<5>(c, a, first_rank, S, tag);
  return run_plain_L<6>(c, a, first_rank, S, tag);
}

}  // namespace cc
