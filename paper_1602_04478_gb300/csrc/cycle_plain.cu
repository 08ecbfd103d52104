// K5 for unannotated root cycles C_L, L = 4, 5, 6 (k = L), heavy sources.
//
// The same DB closure as cycle.cu / cycle_heavy.cu, with the table layout
// fixed by the cycle's shape.  For a source u (highest cycle vertex) and a
// meeting vertex x (image of the node opposite a_0), call the colours other
// than chi(u) and chi(x) the free colours (k - 2 of them):
//   * level 1 (paths u -> v): membership only; v contributes its colour;
//   * level 2 (paths u -> v -> w, L = 5, 6): W2[w][c] = number of lower
//     neighbours v of u adjacent to w with chi(v) = c (chi(w), chi(v),
//     chi(u) distinct), stored as u32 indexed by colour;
//   * at x, over x's neighbours w below u:
//       A[i]    = number of level-1 neighbours w with free colour i
//       M[i][j] = sum of W2[w][free j] over level-2 neighbours w with
//                 free colour i,
//     so the 3-hop half with free colours {i, j} has M[i][j] + M[j][i]
//     matches;
//   * closure (Procedure 2, both halves overlapping only in chi(u), chi(x)):
//       C4: 2 A[0] A[1]
//       C5: sum_i A[i] (M[j][l] + M[l][j]),  {i, j, l} = the free colours
//       C6: 2 sum over the three splits {i,j}|{l,m} of W3[ij] W3[lm].
// Only one highest node is computed (h = 0) and the total is multiplied by L.
// Counts at x are accumulated in registers with predicated updates (the
// free-colour index is data dependent), in 64-bit with overflow checks.
#include <algorithm>

#include "cc_kernels.h"

namespace cc {

constexpr int kPcMaxB = 16;  // sources per heavy group (one lane each per meeting vertex)
constexpr int kPcThreads = 256;

struct PcScratch {
  uint16_t *w2;                // [n][16 sources][8 colours] level-2 rows (u16: max degree < 65536)
  unsigned long long *member;  // [n]: bit b level 1 of source b, bit 32+b level 2 (b < 16)
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
// grid.y = source b; warps walk the lower neighbours v of u_b and their
// neighbours w below u_b.
template <int L>
__global__ void __launch_bounds__(kPcThreads) k_pc_levels(GraphView g, const uint8_t *colors, PcScratch S,
                                                          PcGroup G) {
  const int b = blockIdx.y;
  const int32_t u = G.u[b];
  const int cu = colors[u];
  const int64_t n = g.n;
  const int64_t ub = g.row[u];
  const int du = g.lo_cnt[u];
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp0; i < du; i += nwarps) {
    const int32_t v = __ldg(g.col + ub + i);
    const int cv = colors[v];
    if (cv == cu) continue;
    if (L <= 5 && lane == 0) atomicOr(S.member + v, 1ull << b);
    if (L == 4) continue;
    const int64_t vb = g.row[v];
    const int64_t ve = lower_bound_i32(g.col, vb, g.row[v + 1], u);
    for (int64_t e = vb + lane; e < ve; e += 32) {
      const int32_t w = __ldg(g.col + e);
      const int cw = colors[w];
      if (cw == cu || cw == cv) continue;
      // 16-bit counter inside a 32-bit word; counts stay below 2^16 (host check)
      atomicAdd((uint32_t *)(S.w2 + ((int64_t)w * kPcMaxB + b) * 8 + (cv & ~1)), 1u << (16 * (cv & 1)));
      unsigned long long old = atomicOr(S.member + w, 1ull << (32 + b));
      if (!((old >> (32 + b)) & 1ull)) {
        int slot = atomicAdd(S.cnt + b, 1);
        S.list[(int64_t)b * n + slot] = w;
      }
    }
  }
}

// ---------------------------------- pull ----------------------------------
template <int L>
struct PcAcc {
  u64 A[4];
  u64 M[4][4];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < 4; i++) {
      A[i] = 0;
#pragma unroll
      for (int j = 0; j < 4; j++) M[i][j] = 0;
    }
  }
};

// free-colour index of colour c given the two excluded colours (bit mask ex)
__device__ __forceinline__ int free_idx(int c, uint32_t ex) { return __popc(~ex & ((1u << c) - 1u)); }

template <int L>
__device__ __forceinline__ void pc_visit(PcAcc<L> &acc, const PcScratch &S, int b, int32_t w, int cw,
                                         unsigned long long mem, uint32_t ex, uint32_t fm) {
  if ((ex >> cw) & 1u) return;
  const int fi = free_idx(cw, ex);
  constexpr int F = L - 2;
  if ((L == 4 || L == 5) && ((mem >> b) & 1ull)) {
#pragma unroll
    for (int i = 0; i < F; i++) acc.A[i] += (fi == i) ? 1ull : 0ull;
  }
  if (L >= 5 && ((mem >> (32 + b)) & 1ull)) {
    const uint4 rw = __ldg((const uint4 *)(S.w2 + ((int64_t)w * kPcMaxB + b) * 8));
    const uint32_t words[4] = {rw.x, rw.y, rw.z, rw.w};
    u64 r[4];
    uint32_t rest = fm;  // free colours, ascending
#pragma unroll
    for (int j = 0; j < F; j++) {
      const int c = __ffs(rest) - 1;
      rest &= rest - 1;
      uint32_t wd = (c >> 1) == 0 ? words[0] : (c >> 1) == 1 ? words[1] : (c >> 1) == 2 ? words[2] : words[3];
      r[j] = (wd >> (16 * (c & 1))) & 0xFFFFu;
    }
#pragma unroll
    for (int i = 0; i < F; i++)
#pragma unroll
      for (int j = 0; j < F; j++)
        if (i != j) acc.M[i][j] += (fi == i) ? r[j] : 0ull;
  }
}

template <int L>
__device__ __forceinline__ u64 pc_close(const PcAcc<L> &acc, unsigned &ovf) {
  if (L == 4) return mul_ck(2ull, mul_ck(acc.A[0], acc.A[1], ovf), ovf);
  if (L == 5) {
    u64 t = 0;
    t = add_ck(t, mul_ck(acc.A[0], add_ck(acc.M[1][2], acc.M[2][1], ovf), ovf), ovf);
    t = add_ck(t, mul_ck(acc.A[1], add_ck(acc.M[0][2], acc.M[2][0], ovf), ovf), ovf);
    t = add_ck(t, mul_ck(acc.A[2], add_ck(acc.M[0][1], acc.M[1][0], ovf), ovf), ovf);
    return t;
  }
  u64 w01 = add_ck(acc.M[0][1], acc.M[1][0], ovf), w23 = add_ck(acc.M[2][3], acc.M[3][2], ovf);
  u64 w02 = add_ck(acc.M[0][2], acc.M[2][0], ovf), w13 = add_ck(acc.M[1][3], acc.M[3][1], ovf);
  u64 w03 = add_ck(acc.M[0][3], acc.M[3][0], ovf), w12 = add_ck(acc.M[1][2], acc.M[2][1], ovf);
  u64 t = add_ck(add_ck(mul_ck(w01, w23, ovf), mul_ck(w02, w13, ovf), ovf), mul_ck(w03, w12, ovf), ovf);
  return mul_ck(2ull, t, ovf);
}

// sum a value over the two lanes that share this lane's source (lanes b, b+16)
__device__ __forceinline__ u64 pc_sum4(u64 v, unsigned &ovf) {
  return add_ck(v, __shfl_xor_sync(0xffffffffu, v, 16), ovf);
}

template <int L>
__device__ __forceinline__ void pc_reduce4(PcAcc<L> &acc, unsigned &ovf) {
  constexpr int F = L - 2;
#pragma unroll
  for (int i = 0; i < F; i++) {
    if (L <= 5) acc.A[i] = pc_sum4(acc.A[i], ovf);
#pragma unroll
    for (int j = 0; j < F; j++)
      if (L >= 5 && i != j) acc.M[i][j] = pc_sum4(acc.M[i][j], ovf);
  }
}

// Lane (q, b) of a warp: b = lane & 15 is the source, q = lane >> 4 picks
// one of two meeting vertices (low degree) or half of one vertex's
// neighbours (high degree).  The 16 lanes of a vertex read the same neighbour
// ids and membership words, and adjacent level-2 rows.
template <int L>
__global__ void __launch_bounds__(kPcThreads, 4) k_pc_pull(GraphView g, const uint8_t *colors, PcScratch S, PcGroup G,
                                                        int32_t x_split, int k) {
  const int lane = threadIdx.x & 31;
  const int b = lane & 15, q = lane >> 4;
  const bool active = b < G.B;
  const int32_t ub = active ? G.u[b] : -1;
  const int cu = active ? colors[ub] : 0;
  u64 tot = 0;
  unsigned ovf = 0;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  // low-degree meeting vertices: two per warp
  const int32_t lo_end = min(x_split, G.umax);
  for (int64_t x0 = warp0 * 2; x0 < lo_end; x0 += nwarps * 2) {
    const int32_t x = (int32_t)(x0 + q);
    if (x >= lo_end || !active || x >= ub) continue;
    const int cx = colors[x];
    if (cx == cu) continue;
    const uint32_t ex = (1u << cu) | (1u << cx);
    const uint32_t fm = ~ex & ((1u << k) - 1u);
    PcAcc<L> acc;
    acc.zero();
    const int64_t xb = g.row[x], xe = g.row[x + 1];
    for (int64_t e = xb; e < xe; e++) {
      const int32_t w = __ldg(g.col + e);
      if (w >= ub) break;
      const unsigned long long mem = __ldg(S.member + w);
      if (!((mem >> b) & 0x100000001ull)) continue;
      pc_visit<L>(acc, S, b, w, colors[w], mem, ex, fm);
    }
    tot = add_ck(tot, pc_close<L>(acc, ovf), ovf);
  }
  // high-degree meeting vertices: one warp each, half of the neighbours per lane
  for (int64_t xi = (int64_t)x_split + warp0; xi < G.umax; xi += nwarps) {
    const int32_t x = (int32_t)xi;
    const int cx = colors[x];
    const bool ok = active && x < ub && cx != cu;
    const uint32_t ex = (1u << cu) | (1u << cx);
    const uint32_t fm = ~ex & ((1u << k) - 1u);
    PcAcc<L> acc;
    acc.zero();
    if (ok) {
      const int64_t xb = g.row[x], xe = g.row[x + 1];
      for (int64_t e = xb + q; e < xe; e += 2) {
        const int32_t w = __ldg(g.col + e);
        if (w >= ub) break;
        const unsigned long long mem = __ldg(S.member + w);
        if (!((mem >> b) & 0x100000001ull)) continue;
        pc_visit<L>(acc, S, b, w, colors[w], mem, ex, fm);
      }
    }
    pc_reduce4<L>(acc, ovf);
    if (ok && q == 0) tot = add_ck(tot, pc_close<L>(acc, ovf), ovf);
  }
  tot = pc_sum4(tot, ovf);
  if (q == 0 && active && tot) atomic_add_ck(S.totals + b, tot, ovf);
  (void)ovf;
}

// --------------------------- clear and finish ---------------------------
template <int L>
__global__ void k_pc_clear(GraphView g, const uint8_t *colors, PcScratch S, PcGroup G) {
  const int64_t n = g.n;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nt = (int64_t)gridDim.x * blockDim.x;
  for (int b = 0; b < G.B; b++) {
    const int32_t u = G.u[b];
    const int64_t ub = g.row[u];
    const int du = g.lo_cnt[u];
    for (int64_t i = t0; i < du; i += nt) S.member[__ldg(g.col + ub + i)] = 0;
    if (L >= 5) {
      const int cnt = S.cnt[b];
      for (int64_t i = t0; i < cnt; i += nt) {
        const int32_t w = S.list[(int64_t)b * n + i];
        S.list[(int64_t)b * n + i] = 0;
        S.member[w] = 0;
        *(uint4 *)(S.w2 + ((int64_t)w * kPcMaxB + b) * 8) = make_uint4(0, 0, 0, 0);
      }
    }
  }
  (void)colors;
}

__global__ void k_pc_finish(PcScratch S, PcGroup G, int multiplier, u64 *per_vertex, u64 *status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  unsigned ovf = 0;
  for (int b = 0; b < G.B; b++) {
    u64 t = mul_ck(S.totals[b], (u64)multiplier, ovf);
    S.totals[b] = 0;
    S.cnt[b] = 0;
    if (per_vertex) per_vertex[G.u[b]] = t;
    atomic_add_ck(status + ST_COUNT, t, ovf);
  }
  flag_overflow(status, ovf);
}

// ------------------- light and medium sources: one CTA each -------------------
// Sources of degree below the heavy threshold have small reach sets, so the
// last hop is pushed: every level-2 vertex w adds its row into the level-3
// row of each lower neighbour x (u32, indexed by the unordered pair of free
// colours), and the closure runs over the touched meeting vertices only.
// u32 is exact here: a level-3 entry counts paths u-v-w-x and is at most
// deg(x) * deg(u), which the host checks stays below 2^32.
constexpr int kPlThreads = 256;



__device__ __forceinline__ int pair_idx(int a, int b) {
  int hi = a > b ? a : b, lo = a > b ? b : a;
  return hi * (hi - 1) / 2 + lo;
}

template <int L>
__global__ void __launch_bounds__(kPlThreads) k_pc_light(GraphView g, const uint8_t *colors, PlScratch S,
                                                         int32_t end_rank, int *work, int multiplier,
                                                         u64 *per_vertex, u64 *status, int k) {
  __shared__ int s_u, s_n2, s_n3;
  __shared__ unsigned long long s_tot;
  __shared__ unsigned s_ovf;
  char *slot = S.base + (size_t)blockIdx.x * S.slot_bytes;
  uint32_t *W2 = (uint32_t *)(slot + S.o_w2);   // [n][8] by colour
  uint32_t *W3 = (uint32_t *)(slot + S.o_w3);   // [n][16] by colour pair
  uint32_t *mark = (uint32_t *)(slot + S.o_mark);
  int32_t *L2 = (int32_t *)(slot + S.o_l2);
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
    unsigned ovf = 0;
    if (du >= 2) {
      // level 2: W2[w][chi(v)] over v in N<(u), w in N<u(v)
      for (int i = wib; i < du; i += NW) {
        const int32_t v = __ldg(g.col + ub + i);
        const int cv = colors[v];
        if (cv == cu) continue;
        const int64_t vb = g.row[v];
        const int64_t ve = lower_bound_i32(g.col, vb, g.row[v + 1], u);
        for (int64_t e = vb + lane; e < ve; e += 32) {
          const int32_t w = __ldg(g.col + e);
          const int cw = colors[w];
          if (cw == cu || cw == cv) continue;
          atomicAdd(W2 + (int64_t)w * 8 + cv, 1u);
          if (!(atomicOr(mark + w, 1u) & 1u)) L2[atomicAdd(&s_n2, 1)] = w;
        }
      }
      __syncthreads();
      const int n2 = s_n2;
      if (L >= 5) {
        // level 3 pushed into the pair rows of the meeting vertices x
        for (int i = wib; i < n2; i += NW) {
          const int32_t w = L2[i];
          const int cw = colors[w];
          const uint4 r0 = *(const uint4 *)(W2 + (int64_t)w * 8);
          const uint4 r1 = *(const uint4 *)(W2 + (int64_t)w * 8 + 4);
          const uint32_t row[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
          const int64_t wb = g.row[w];
          const int64_t we = lower_bound_i32(g.col, wb, g.row[w + 1], u);
          for (int64_t e = wb + lane; e < we; e += 32) {
            const int32_t x = __ldg(g.col + e);
            const int cx = colors[x];
            if (cx == cu || cx == cw) continue;
            bool any = false;
#pragma unroll
            for (int c = 0; c < 8; c++) {
              const uint32_t t = row[c];
              if (!t || c == cx) continue;
              atomicAdd(W3 + (int64_t)x * 16 + pair_idx(cw, c), t);
              any = true;
            }
            if (any && !(atomicOr(mark + x, 2u) & 2u)) L3[atomicAdd(&s_n3, 1)] = x;
          }
        }
        __syncthreads();
      }
      // closure at the meeting vertices
      const int nx = L >= 5 ? s_n3 : n2;
      const int32_t *LX = L >= 5 ? L3 : L2;
      u64 mine = 0;
      for (int i = tid; i < nx; i += kPlThreads) {
        const int32_t x = LX[i];
        if (L >= 5) L3[i] = 0;  // lists are cleared as they are consumed
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
          const u64 a0 = W2[(int64_t)x * 8 + f[0]], a1 = W2[(int64_t)x * 8 + f[1]];
          mine = add_ck(mine, mul_ck(2ull, mul_ck(a0, a1, ovf), ovf), ovf);
        } else if (L == 5) {
          const uint32_t *w3 = W3 + (int64_t)x * 16;
          const uint32_t *w2 = W2 + (int64_t)x * 8;
          u64 t = mul_ck((u64)w2[f[0]], (u64)w3[pair_idx(f[1], f[2])], ovf);
          t = add_ck(t, mul_ck((u64)w2[f[1]], (u64)w3[pair_idx(f[0], f[2])], ovf), ovf);
          t = add_ck(t, mul_ck((u64)w2[f[2]], (u64)w3[pair_idx(f[0], f[1])], ovf), ovf);
          mine = add_ck(mine, t, ovf);
        } else {
          const uint32_t *w3 = W3 + (int64_t)x * 16;
          u64 t = mul_ck((u64)w3[pair_idx(f[0], f[1])], (u64)w3[pair_idx(f[2], f[3])], ovf);
          t = add_ck(t, mul_ck((u64)w3[pair_idx(f[0], f[2])], (u64)w3[pair_idx(f[1], f[3])], ovf), ovf);
          t = add_ck(t, mul_ck((u64)w3[pair_idx(f[0], f[3])], (u64)w3[pair_idx(f[1], f[2])], ovf), ovf);
          mine = add_ck(mine, mul_ck(2ull, t, ovf), ovf);
        }
        if (L >= 5) {
          uint4 *z = (uint4 *)(W3 + (int64_t)x * 16);
          z[0] = z[1] = z[2] = z[3] = make_uint4(0, 0, 0, 0);
          atomicAnd(mark + x, ~2u);
        }
      }
      mine = warp_sum_ck(mine, ovf);
      if (lane == 0 && mine) {
        unsigned long long old = atomicAdd(&s_tot, mine);
        if (old + mine < old) ovf = 1;
      }
      __syncthreads();
      for (int i = tid; i < n2; i += kPlThreads) {
        const int32_t w = L2[i];
        L2[i] = 0;
        uint4 *z = (uint4 *)(W2 + (int64_t)w * 8);
        z[0] = z[1] = make_uint4(0, 0, 0, 0);
        atomicAnd(mark + w, ~1u);
      }
    }
    if (ovf) atomicOr(&s_ovf, 1u);
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
  S.o_l2 = take((size_t)n * 4);
  S.o_l3 = a.L >= 5 ? take((size_t)n * 4) : 0;
  S.slot_bytes = off;
  size_t budget = c.budget ? (c.budget > c.in_use ? (c.budget - c.in_use) / 2 : 0) : ((size_t)16 << 30);
  int slots = (int)std::min<size_t>(152 * 2, budget / std::max<size_t>(1, S.slot_bytes));
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

template <int L>
static int run_plain_L(Ctx &c, const CycleArgs &a, int32_t first_rank, int32_t x_split, const PcScratch &S) {
  const int64_t n = a.g.n;
  const int sms = 152;
  for (int64_t top = n - 1; top >= first_rank; top -= kPcMaxB) {
    PcGroup G;
    G.B = (int)std::min<int64_t>(kPcMaxB, top - first_rank + 1);
    G.umax = (int32_t)top;
    for (int b = 0; b < G.B; b++) G.u[b] = (int32_t)(top - b);
    int64_t du = c.cur_graph_row[top + 1] - c.cur_graph_row[top];
    dim3 gl((unsigned)std::max<int64_t>(1, std::min<int64_t>(sms * 2, (du * 32 + kPcThreads - 1) / kPcThreads)),
            G.B);
    timing_begin(c, "cycle_plain_levels");
    k_pc_levels<L><<<gl, kPcThreads, 0, c.stream>>>(a.g, a.colors, S, G);
    c.kernels++;
    timing_end(c);
    timing_begin(c, "cycle_plain_pull");
    k_pc_pull<L><<<sms * 4, kPcThreads, 0, c.stream>>>(a.g, a.colors, S, G, x_split, a.k);
    c.kernels++;
    timing_end(c);
    k_pc_clear<L><<<sms, 256, 0, c.stream>>>(a.g, a.colors, S, G);
    c.kernels++;
    k_pc_finish<<<1, 32, 0, c.stream>>>(S, G, a.multiplier, a.per_vertex, a.status);
    c.kernels++;
  }
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
  size_t o_w2 = lv2 ? take((size_t)kPcMaxB * n * 8 * 2) : 0;
  size_t o_mem = take((size_t)n * 8);
  size_t o_list = lv2 ? take((size_t)kPcMaxB * n * 4) : 0;
  size_t o_cnt = take(kPcMaxB * 4);
  size_t o_tot = take(kPcMaxB * 8);
  size_t need = off;
  int rc0 = ensure_hv_scratch(c, need);
  if (rc0 != CC_OK) return rc0;
  char *base = (char *)c.hv_scratch;
  PcScratch S;
  S.w2 = (uint16_t *)(base + o_w2);
  S.member = (unsigned long long *)(base + o_mem);
  S.list = (int32_t *)(base + o_list);
  S.cnt = (int *)(base + o_cnt);
  S.totals = (u64 *)(base + o_tot);
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) / 2;
    if (c.cur_graph_row[mid + 1] - c.cur_graph_row[mid] >= 32) hi = mid;
    else lo = mid + 1;
  }
  const int32_t x_split = (int32_t)lo;
  if (a.L == 4) return run_plain_L<4>(c, a, first_rank, x_split, S);
  if (a.L == 5) return run_plain_L<5>(c, a, first_rank, x_split, S);
  return run_plain_L<6>(c, a, first_rank, x_split, S);
}

}  // namespace cc
