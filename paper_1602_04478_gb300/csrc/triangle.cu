// K3: triangle blocks (cycle blocks of length 3).
//
// A triangle block (a0, a1, a2) may be annotated on its nodes (unary tables)
// and edges (edge-keyed tables) and has 0 (root), 1 (Case 1) or 2 (Case 2)
// boundary nodes.  By Eq. 1 its colourful matches split by which query node
// takes the highest data vertex; here every data triangle {u > v > w} is
// listed once from its highest vertex u (the MinBucket order the paper
// generalises: u scans its lower neighbours v and, for each, v's lower
// neighbours w that are also lower neighbours of u), and all six
// assignments of (a0, a1, a2) to (u, v, w) are joined with the annotating
// tables:
//   value = prod N_i[p_i][S_i] * prod E_i[(p_i, p_i+1)][T_i]
// over signatures that overlap exactly in the colours of shared vertices;
// the union is the block's signature.  The result is added to the output
// row of the boundary image(s) (unary row, or the directed-edge row of the
// boundary pair, which is a data edge because triangle nodes are pairwise
// adjacent), or to the root count.
//
// Two kernels share the per-triangle work:
//  * k_triangle_hub, one CTA per source u of degree >= kHubDegree: the CTA
//    puts N<(u) into a shared-memory hash set (open addressing, at most half
//    full), then its warps scan the wedges (v, w) and test w against the set
//    in O(1); contributions to u's own output row gather in shared memory and
//    reach the table once per source.  On skewed graphs these sources hold
//    almost all wedges.
//  * k_triangle, one warp per remaining source, w tested by binary search in
//    the sorted N<(u).
// A wedge whose first two vertices share a colour cannot close a colourful
// triangle, so v with chi(v) = chi(u) is skipped before its list is read.
#include <algorithm>
#include <vector>

#include "cc_kernels.h"

namespace cc {

constexpr int kMaxPartial = 128;
constexpr int kHubDegree = 32;        // sources of at least this degree take the CTA kernel
constexpr int kHubMaxSlots = 16384;   // hash slots per CTA (N<(u) of up to 8192 vertices)
constexpr int kHubThreads = 256;

struct TriEdges {
  int64_t pos[3][3];  // pos[i][j]: CSR position of directed edge p_i -> p_j (local ids 0=u,1=v,2=w)
};

// Where unary contributions go: the output table, except those to vertex u
// when the caller gathers u's row in shared memory (acc != nullptr).
struct USink {
  int32_t u = -1;
  u64 *acc = nullptr;
};

__device__ __forceinline__ void emit_unary(const TriArgs &a, const USink &sk, int32_t x, int slot, u64 v,
                                           unsigned &ovf) {
  if (x == sk.u) atomic_add_ck(sk.acc + slot, v, ovf);
  else atomic_add_ck(a.out + (int64_t)x * a.R_out + slot, v, ovf);
}

__device__ void tri_emit_plain(const TriArgs &a, const USink &sk, const int32_t vx[3], const int c[3],
                               const TriEdges &te, u64 &root_acc, unsigned &ovf) {
  uint32_t S = (1u << c[0]) | (1u << c[1]) | (1u << c[2]);
  if (a.nb == 0) {
    root_acc = add_ck(root_acc, 6ull, ovf);
  } else if (a.nb == 1) {
#pragma unroll
    for (int i = 0; i < 3; i++) emit_unary(a, sk, vx[i], uslot(a.lut, S, c[i]), 2ull, ovf);
  } else {
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
      for (int j = 0; j < 3; j++)
        if (i != j) atomic_add_ck(a.out + te.pos[i][j] * a.R_out + pslot(a.lut, S, c[i], c[j]), 1ull, ovf);
  }
}

// join a partial list with one table row: keep pairs whose masks overlap in
// exactly `shared`, merge equal result masks
__device__ int tri_join(uint16_t *pm, u64 *pv, int np, const u64 *row, int R, int s, bool pair, int ca,
                        int cb, uint32_t shared, const Lut &lut, unsigned &ovf) {
  uint16_t nm[kMaxPartial];
  u64 nv[kMaxPartial];
  int nn = 0;
  for (int j = 0; j < R; j++) {
    u64 t = __ldg(row + j);
    if (!t) continue;
    uint32_t mt = pair ? pmask(lut, s, j, ca, cb) : umask(lut, s, j, ca);
    for (int q = 0; q < np; q++) {
      if ((pm[q] & mt) != shared) continue;
      uint16_t m = (uint16_t)(pm[q] | mt);
      u64 v = mul_ck(pv[q], t, ovf);
      int f = 0;
      while (f < nn && nm[f] != m) f++;
      if (f == nn) {
        if (nn == kMaxPartial) { ovf |= 2u; continue; }
        nm[nn] = m;
        nv[nn] = 0;
        nn++;
      }
      nv[f] = add_ck(nv[f], v, ovf);
    }
  }
  for (int q = 0; q < nn; q++) pm[q] = nm[q], pv[q] = nv[q];
  return nn;
}

__device__ void tri_emit_general(const TriArgs &a, const USink &sk, const int32_t vx[3], const int c[3],
                                 const TriEdges &te, u64 &root_acc, unsigned &ovf) {
  // all six assignments (a0, a1, a2) -> local vertices (perm[0], perm[1], perm[2])
  const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  for (int pi = 0; pi < 6; pi++) {
    const int *p = perms[pi];
    int cc0 = c[p[0]], cc1 = c[p[1]], cc2 = c[p[2]];
    uint16_t pm[kMaxPartial];
    u64 pv[kMaxPartial];
    pm[0] = (uint16_t)((1u << cc0) | (1u << cc1) | (1u << cc2));
    pv[0] = 1;
    int np = 1;
    for (int i = 0; i < 3 && np > 0; i++) {
      if (!a.N[i].p) continue;
      int ci = c[p[i]];
      np = tri_join(pm, pv, np, a.N[i].p + (int64_t)vx[p[i]] * a.N[i].R, a.N[i].R, a.N[i].s, false, ci, 0,
                    1u << ci, a.lut, ovf);
    }
    for (int i = 0; i < 3 && np > 0; i++) {
      if (!a.E[i].p) continue;
      int li = p[i], lj = p[(i + 1) % 3];
      int64_t e = a.E[i].use_rev ? te.pos[lj][li] : te.pos[li][lj];
      int ci = c[li], cj = c[lj];
      np = tri_join(pm, pv, np, a.E[i].p + e * a.E[i].R, a.E[i].R, a.E[i].s, true, ci, cj,
                    (1u << ci) | (1u << cj), a.lut, ovf);
    }
    for (int q = 0; q < np; q++) {
      if (!pv[q]) continue;
      if (a.nb == 0) {
        root_acc = add_ck(root_acc, pv[q], ovf);
      } else if (a.nb == 1) {
        int lb = p[a.bd[0]];
        emit_unary(a, sk, vx[lb], uslot(a.lut, pm[q], c[lb]), pv[q], ovf);
      } else {
        int l0 = p[a.bd[0]], l1 = p[a.bd[1]];
        atomic_add_ck(a.out + te.pos[l0][l1] * a.R_out + pslot(a.lut, pm[q], c[l0], c[l1]), pv[q], ovf);
      }
    }
  }
}

// x[i] for a runtime i in 0..2 without indexing a local array
template <class T>
__device__ __forceinline__ T pick3(const T x[3], int i) {
  return i == 0 ? x[0] : (i == 1 ? x[1] : x[2]);
}
// te.pos[i][j] for runtime i != j
__device__ __forceinline__ int64_t tpos(const TriEdges &te, int i, int j) {
  return i == 0 ? (j == 1 ? te.pos[0][1] : te.pos[0][2])
                : (i == 1 ? (j == 0 ? te.pos[1][0] : te.pos[1][2]) : (j == 0 ? te.pos[2][0] : te.pos[2][1]));
}

// One annotation only (a node table at position ai, or an edge table on edge
// ai -> ai+1): each of its row's signatures extends the triangle's colours
// directly, without partial lists.
__device__ __forceinline__ void tri_emit_one(const TriArgs &a, const USink &sk, const int32_t vx[3], const int c[3],
                                             const TriEdges &te, u64 &root_acc, unsigned &ovf, int ai, bool edge) {
  const uint32_t K = (1u << a.k) - 1u;
  const uint32_t base = (1u << c[0]) | (1u << c[1]) | (1u << c[2]);
  if (a.nb == 0 && !edge) {
    // root, one node table: the signature is the full colour set, so the
    // value of an assignment depends only on which vertex takes a_ai, and
    // each vertex takes it in two of the six assignments
    const TabU &N = a.N[ai];
    u64 t = 0;
#pragma unroll
    for (int x = 0; x < 3; x++)
      t = add_ck(t, __ldg(N.p + (int64_t)vx[x] * N.R + uslot(a.lut, (K & ~base) | (1u << c[x]), c[x])), ovf);
    root_acc = add_ck(root_acc, add_ck(t, t, ovf), ovf);
    return;
  }
  const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
#pragma unroll
  for (int pi = 0; pi < 6; pi++) {
    const int *p = perms[pi];
    const int li = pick3(p, ai), lj = pick3(p, ai == 2 ? 0 : ai + 1);
    const int cli = pick3(c, li), clj = pick3(c, lj);
    const u64 *row;
    int R, s;
    uint32_t shared;
    if (edge) {
      const TabE &E = a.E[ai];
      int64_t e = E.use_rev ? tpos(te, lj, li) : tpos(te, li, lj);
      row = E.p + e * E.R;
      R = E.R;
      s = E.s;
      shared = (1u << cli) | (1u << clj);
    } else {
      const TabU &N = a.N[ai];
      row = N.p + (int64_t)pick3(vx, li) * N.R;
      R = N.R;
      s = N.s;
      shared = 1u << cli;
    }
    if (a.nb == 0) {
      uint32_t m = (K & ~base) | shared;
      int slot = edge ? pslot(a.lut, m, cli, clj) : uslot(a.lut, m, cli);
      root_acc = add_ck(root_acc, __ldg(row + slot), ovf);
      continue;
    }
    const int lb = pick3(p, a.bd[0]);
    const int lb1 = a.nb == 2 ? pick3(p, a.bd[1]) : lb;
    for (int j = 0; j < R; j++) {
      u64 t = __ldg(row + j);
      if (!t) continue;
      uint32_t mt = edge ? pmask(a.lut, s, j, cli, clj) : umask(a.lut, s, j, cli);
      if ((mt & base) != shared) continue;
      uint32_t m = mt | base;
      if (a.nb == 1) {
        emit_unary(a, sk, pick3(vx, lb), uslot(a.lut, m, pick3(c, lb)), t, ovf);
      } else {
        atomic_add_ck(a.out + tpos(te, lb, lb1) * a.R_out + pslot(a.lut, m, pick3(c, lb), pick3(c, lb1)), t, ovf);
      }
    }
  }
}

// How the kernels emit a listed triangle: which of the forms above, and
// whether the directed-edge positions are needed (edge tables or an
// edge-keyed output).
struct TriMode {
  bool plain = true;
  int one_pos = -1;
  bool one_edge = false;
  bool need_pos = false;
};

// One colourful triangle u > v > w: u->v at CSR position p01, u->w at p02,
// v->w at p12.  kForm: 0 plain, 1 one annotation, 2 general.
template <int kForm>
__device__ __forceinline__ void tri_visit(const TriArgs &a, const TriMode &md, const USink &sk, int32_t u,
                                          int32_t v, int32_t w, int cu, int cv, int cw, int64_t p01, int64_t p02,
                                          int64_t p12, u64 &root_acc, unsigned &ovf) {
  int32_t vx[3] = {u, v, w};
  int c[3] = {cu, cv, cw};
  TriEdges te;
  if (md.need_pos) {
    te.pos[0][1] = p01;
    te.pos[0][2] = p02;
    te.pos[1][2] = p12;
    te.pos[1][0] = __ldg(a.g.rev + p01);
    te.pos[2][0] = __ldg(a.g.rev + p02);
    te.pos[2][1] = __ldg(a.g.rev + p12);
    te.pos[0][0] = te.pos[1][1] = te.pos[2][2] = -1;
  }
  if (kForm == 0) tri_emit_plain(a, sk, vx, c, te, root_acc, ovf);
  else if (kForm == 1) tri_emit_one(a, sk, vx, c, te, root_acc, ovf, md.one_pos, md.one_edge);
  else tri_emit_general(a, sk, vx, c, te, root_acc, ovf);
}

// One warp per source u in [0, u_end), highest first.
template <int kForm>
__global__ void __launch_bounds__(256) k_triangle(TriArgs a, TriMode md, int32_t u_end) {
  const int lane = threadIdx.x & 31;
  USink sk;
  unsigned ovf = 0;
  while (true) {
    int idx = 0;
    if (lane == 0) idx = atomicAdd(a.work_counter, 1);
    idx = __shfl_sync(0xffffffffu, idx, 0);
    if (idx >= u_end) break;
    const int32_t u = u_end - 1 - idx;
    const int64_t ub = a.g.row[u];
    const int du = a.g.lo_cnt[u];
    const int cu = a.colors[u];
    u64 root_acc = 0;
    u64 units = 0;
    for (int iv = 1; iv < du; iv++) {
      const int32_t v = __ldg(a.g.col + ub + iv);
      const int dv = a.g.lo_cnt[v];
      units += (u64)dv;
      const int cv = a.colors[v];
      if (cv == cu) continue;
      const int64_t vb = a.g.row[v];
      for (int j = lane; j < dv; j += 32) {
        const int32_t w = __ldg(a.g.col + vb + j);
        // w < v is a lower neighbour of u: search N<(u)[0, iv)
        int64_t p = lower_bound_i32(a.g.col, ub, ub + iv, w);
        if (p >= ub + iv || __ldg(a.g.col + p) != w) continue;
        const int cw = a.colors[w];
        // a colourful match maps the triangle to three distinct colours
        if (cu == cw || cv == cw) continue;
        tri_visit<kForm>(a, md, sk, u, v, w, cu, cv, cw, ub + iv, p, vb + j, root_acc, ovf);
      }
    }
    if (a.count_units && lane == 0 && units) atomicAdd(a.status + ST_UNITS, units);
    if (a.nb == 0) {
      root_acc = warp_sum_ck(root_acc, ovf);
      if (lane == 0 && root_acc) {
        atomic_add_ck(a.status + ST_COUNT, root_acc, ovf);
        if (a.per_vertex) a.per_vertex[u] = root_acc;
      }
    }
  }
  flag_overflow(a.status, ovf & 1u);
  if (ovf & 2u) atomicOr(a.status + ST_TIMEOUT, 2ull);  // partial list capacity exceeded
}

__device__ __forceinline__ uint32_t hub_hash(int32_t w) { return (uint32_t)w * 0x9E3779B1u; }

// One CTA per source u in [u_lo, n), highest first.  Shared memory:
//   acc[R_acc]        u's output row (unary output only), all zero between sources
//   keys[max_slots]   hash set of N<(u) (-1 = empty), all empty between sources
//   kpos[max_slots]   index of the key in N<(u) (only when positions are needed)
// A source with |N<(u)| > max_slots / 2 scans by binary search instead.
template <int kForm>
__global__ void __launch_bounds__(kHubThreads) k_triangle_hub(TriArgs a, TriMode md, int32_t u_lo, int max_slots,
                                                              int R_acc) {
  extern __shared__ __align__(16) unsigned char smem[];
  u64 *acc = reinterpret_cast<u64 *>(smem);
  int32_t *keys = reinterpret_cast<int32_t *>(smem + (size_t)R_acc * 8);
  uint16_t *kpos = reinterpret_cast<uint16_t *>(keys + max_slots);
  __shared__ int s_idx;
  __shared__ u64 s_root;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  unsigned ovf = 0;
  for (int i = tid; i < max_slots; i += blockDim.x) keys[i] = -1;
  for (int i = tid; i < R_acc; i += blockDim.x) acc[i] = 0;
  if (tid == 0) s_root = 0;
  const int32_t n_hub = (int32_t)(a.g.n - u_lo);
  while (true) {
    __syncthreads();  // readers of s_idx and the previous source's clean-up are done
    if (tid == 0) s_idx = atomicAdd(a.work_counter, 1);
    __syncthreads();
    const int idx = s_idx;
    if (idx >= n_hub) break;
    const int32_t u = (int32_t)(a.g.n - 1 - idx);
    const int64_t ub = a.g.row[u];
    const int du = a.g.lo_cnt[u];
    if (du < 2) continue;
    const int cu = a.colors[u];
    const bool hashed = 2 * du <= max_slots;
    int slots = 64;
    if (hashed)
      while (slots < 2 * du) slots <<= 1;
    const uint32_t mask = (uint32_t)slots - 1u;
    const int shift = 32 - __ffs(slots) + 1;  // top log2(slots) bits of the hash
    if (hashed) {
      for (int i = tid; i < du; i += blockDim.x) {
        const int32_t w = __ldg(a.g.col + ub + i);
        uint32_t h = hub_hash(w) >> shift;
        for (int t = 0; t < slots; t++, h = (h + 1u) & mask) {
          if (atomicCAS(keys + h, -1, w) == -1) {
            if (md.need_pos) kpos[h] = (uint16_t)i;
            break;
          }
        }
      }
      __syncthreads();
    }
    USink sk;
    if (a.nb == 1) sk.u = u, sk.acc = acc;
    u64 root_acc = 0, units = 0;
    for (int iv = 1 + warp; iv < du; iv += nwarps) {
      const int32_t v = __ldg(a.g.col + ub + iv);
      const int dv = a.g.lo_cnt[v];
      units += (u64)dv;
      const int cv = a.colors[v];
      if (cv == cu) continue;
      const int64_t vb = a.g.row[v];
      for (int j = lane; j < dv; j += 32) {
        const int32_t w = __ldg(a.g.col + vb + j);
        int64_t p = -1;
        if (hashed) {
          uint32_t h = hub_hash(w) >> shift;
          for (int t = 0; t < slots; t++, h = (h + 1u) & mask) {
            const int32_t kk = keys[h];
            if (kk == w) {
              p = md.need_pos ? ub + kpos[h] : 0;
              break;
            }
            if (kk < 0) break;
          }
          if (p < 0) continue;
        } else {
          p = lower_bound_i32(a.g.col, ub, ub + iv, w);
          if (p >= ub + iv || __ldg(a.g.col + p) != w) continue;
        }
        const int cw = a.colors[w];
        if (cu == cw || cv == cw) continue;
        tri_visit<kForm>(a, md, sk, u, v, w, cu, cv, cw, ub + iv, p, vb + j, root_acc, ovf);
      }
    }
    if (a.count_units && lane == 0 && units) atomicAdd(a.status + ST_UNITS, units);
    if (a.nb == 0) {
      root_acc = warp_sum_ck(root_acc, ovf);
      if (lane == 0 && root_acc) atomic_add_ck(&s_root, root_acc, ovf);
    }
    __syncthreads();
    if (a.nb == 0 && tid == 0) {
      const u64 r = s_root;
      if (r) {
        atomic_add_ck(a.status + ST_COUNT, r, ovf);
        if (a.per_vertex) a.per_vertex[u] = r;
      }
      s_root = 0;
    }
    if (a.nb == 1) {
      for (int i = tid; i < R_acc; i += blockDim.x) {
        const u64 t = acc[i];
        if (t) {
          atomic_add_ck(a.out + (int64_t)u * a.R_out + i, t, ovf);
          acc[i] = 0;
        }
      }
    }
    if (hashed)
      for (int i = tid; i < slots; i += blockDim.x) keys[i] = -1;
  }
  flag_overflow(a.status, ovf & 1u);
  if (ovf & 2u) atomicOr(a.status + ST_TIMEOUT, 2ull);  // partial list capacity exceeded
}

// ------------------------------ triangle list ------------------------------
// The triangles of a graph do not depend on the colouring.  They are listed
// once (the same MinBucket enumeration as above: u scans its lower
// neighbours v, and v's lower neighbours w are tested against N<(u)), into
// arrays grouped by u; every colouring then streams the list and only checks
// colours and emits, instead of re-scanning about 20 wedges per triangle.
//
// Listing runs twice: the first pass counts each source's triangles, the
// host turns the counts into offsets, the second pass writes them.
constexpr int kListHubDegree = 64;  // sources with at least this many lower neighbours: one CTA each

// one warp per source u of [0, u_end) with fewer than kListHubDegree lower neighbours
template <bool kWrite>
__global__ void k_tl_warp(GraphView g, int32_t u_end, int64_t *counts, const int64_t *offs, int32_t *tu,
                          int32_t *tv, int32_t *tw, int64_t *tp, int64_t n_tri) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t ui = warp0; ui < u_end; ui += nwarps) {
    const int32_t u = (int32_t)ui;
    const int64_t ub = g.row[u];
    const int du = g.lo_cnt[u];
    if (du >= kListHubDegree) continue;
    int64_t at = kWrite ? offs[u] : 0;
    for (int iv = 1; iv < du; iv++) {
      const int32_t v = __ldg(g.col + ub + iv);
      const int64_t vb = g.row[v];
      const int dv = g.lo_cnt[v];
      for (int j0 = 0; j0 < dv; j0 += 32) {
        const int j = j0 + lane;
        int64_t p = -1;
        if (j < dv) {
          const int32_t w = __ldg(g.col + vb + j);
          const int64_t q = lower_bound_i32(g.col, ub, ub + iv, w);
          if (q < ub + iv && __ldg(g.col + q) == w) p = q;
        }
        const unsigned hit = __ballot_sync(FULL, p >= 0);
        if (kWrite && p >= 0) {
          const int64_t i = at + __popc(hit & ((1u << lane) - 1u));
          tu[i] = u;
          tv[i] = v;
          tw[i] = __ldg(g.col + p);
          tp[i] = ub + iv;
          tp[n_tri + i] = p;
          tp[2 * n_tri + i] = vb + j;
        }
        at += __popc(hit);
      }
    }
    if (!kWrite && lane == 0) counts[u] = at;
  }
}

// one CTA per source u of [0, u_end) with at least kListHubDegree lower
// neighbours (work counter, highest first): N<(u) in a shared-memory hash set
// with each key's index, or binary search when it does not fit
template <bool kWrite>
__global__ void __launch_bounds__(kHubThreads) k_tl_hub(GraphView g, int32_t u_end, int *work, int max_slots,
                                                        int64_t *counts, const int64_t *offs, int32_t *tu,
                                                        int32_t *tv, int32_t *tw, int64_t *tp, int64_t n_tri) {
  constexpr unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(16) unsigned char tl_smem[];
  int32_t *keys = reinterpret_cast<int32_t *>(tl_smem);
  int32_t *kpos = keys + max_slots;
  __shared__ int s_idx;
  __shared__ unsigned long long s_at;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  for (int i = tid; i < max_slots; i += blockDim.x) keys[i] = -1;
  while (true) {
    __syncthreads();
    if (tid == 0) s_idx = atomicAdd(work, 1);
    __syncthreads();
    const int idx = s_idx;
    if (idx >= u_end) break;
    const int32_t u = u_end - 1 - idx;
    const int64_t ub = g.row[u];
    const int du = g.lo_cnt[u];
    if (du < kListHubDegree) continue;
    if (tid == 0) s_at = kWrite ? (unsigned long long)offs[u] : 0ull;
    const bool hashed = 2 * du <= max_slots;
    int slots = 64;
    if (hashed)
      while (slots < 2 * du) slots <<= 1;
    const uint32_t mask = (uint32_t)slots - 1u;
    const int shift = 32 - __ffs(slots) + 1;
    if (hashed) {
      for (int i = tid; i < du; i += blockDim.x) {
        const int32_t w = __ldg(g.col + ub + i);
        uint32_t h = hub_hash(w) >> shift;
        for (int t = 0; t < slots; t++, h = (h + 1u) & mask)
          if (atomicCAS(keys + h, -1, w) == -1) {
            kpos[h] = i;
            break;
          }
      }
    }
    __syncthreads();
    for (int iv = 1 + warp; iv < du; iv += nwarps) {
      const int32_t v = __ldg(g.col + ub + iv);
      const int64_t vb = g.row[v];
      const int dv = g.lo_cnt[v];
      for (int j0 = 0; j0 < dv; j0 += 32) {
        const int j = j0 + lane;
        int64_t p = -1;
        if (j < dv) {
          const int32_t w = __ldg(g.col + vb + j);
          if (hashed) {
            uint32_t h = hub_hash(w) >> shift;
            for (int t = 0; t < slots; t++, h = (h + 1u) & mask) {
              const int32_t kk = keys[h];
              if (kk == w) {
                p = ub + kpos[h];
                break;
              }
              if (kk < 0) break;
            }
          } else {
            const int64_t q = lower_bound_i32(g.col, ub, ub + iv, w);
            if (q < ub + iv && __ldg(g.col + q) == w) p = q;
          }
        }
        const unsigned hit = __ballot_sync(FULL, p >= 0);
        if (!hit) continue;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&s_at, (unsigned long long)__popc(hit));
        base = __shfl_sync(FULL, base, 0);
        if (kWrite && p >= 0) {
          const int64_t i = (int64_t)base + __popc(hit & ((1u << lane) - 1u));
          tu[i] = u;
          tv[i] = v;
          tw[i] = __ldg(g.col + p);
          tp[i] = ub + iv;
          tp[n_tri + i] = p;
          tp[2 * n_tri + i] = vb + j;
        }
      }
    }
    __syncthreads();
    if (!kWrite && tid == 0) counts[u] = (int64_t)s_at;
    if (hashed)
      for (int i = tid; i < slots; i += blockDim.x) keys[i] = -1;
  }
}

void tri_list_free(Ctx &c, DevGraph &g) {
  if (g.tri_state == 1 && g.owned) {
    const size_t n = (size_t)std::max<int64_t>(g.n_tri, 1);
    dev_free(c, g.tri_u, n * 4);
    dev_free(c, g.tri_v, n * 4);
    dev_free(c, g.tri_w, n * 4);
    dev_free(c, g.tri_p, n * 24);
  }
  g.tri_u = g.tri_v = g.tri_w = nullptr;
  g.tri_p = nullptr;
  g.n_tri = 0;
  g.tri_state = 0;
}

static int tl_launch(Ctx &c, const GraphView &gv, bool write, int64_t *counts, const int64_t *offs, int32_t *tu,
                     int32_t *tv, int32_t *tw, int64_t *tp, int64_t n_tri, int *work, int max_slots, size_t smem) {
  const int32_t n = (int32_t)gv.n;
  if (cudaMemsetAsync(work, 0, sizeof(int), c.stream) != cudaSuccess) return CC_ERR_CUDA;
  if (write) {
    k_tl_warp<true><<<152 * 8, 256, 0, c.stream>>>(gv, n, counts, offs, tu, tv, tw, tp, n_tri);
    k_tl_hub<true><<<152 * 2, kHubThreads, smem, c.stream>>>(gv, n, work, max_slots, counts, offs, tu, tv, tw, tp,
                                                             n_tri);
  } else {
    k_tl_warp<false><<<152 * 8, 256, 0, c.stream>>>(gv, n, counts, offs, tu, tv, tw, tp, n_tri);
    k_tl_hub<false><<<152 * 2, kHubThreads, smem, c.stream>>>(gv, n, work, max_slots, counts, offs, tu, tv, tw, tp,
                                                              n_tri);
  }
  c.kernels += 2;
  return cudaGetLastError() == cudaSuccess ? CC_OK : CC_ERR_CUDA;
}

int tri_list_build(Ctx &c, DevGraph &g) {
  if (g.tri_state != 0) return CC_OK;
  const int64_t n = g.n;
  GraphView gv = view_of(g);
  int max_slots = 64;
  while (max_slots < kHubMaxSlots && max_slots < 2 * g.max_deg) max_slots <<= 1;
  const size_t smem = (size_t)max_slots * 8;
  if (smem > 48 * 1024) {
    if (cudaFuncSetAttribute(k_tl_hub<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(k_tl_hub<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return CC_ERR_CUDA;
  }
  int64_t *counts = (int64_t *)dev_alloc(c, (size_t)(n + 1) * 8);
  int *work = (int *)dev_alloc(c, 256);
  if (!counts || !work) {
    dev_free(c, counts, (size_t)(n + 1) * 8);
    dev_free(c, work, 256);
    return CC_ERR_OOM;
  }
  int rc = CC_OK;
  std::vector<int64_t> h((size_t)n + 1, 0);
  timing_begin(c, "triangle_list_build");
  do {
    if ((rc = tl_launch(c, gv, false, counts, nullptr, nullptr, nullptr, nullptr, nullptr, 0, work, max_slots,
                        smem)) != CC_OK)
      break;
    if (cudaMemcpyAsync(h.data(), counts, (size_t)n * 8, cudaMemcpyDeviceToHost, c.stream) != cudaSuccess ||
        cudaStreamSynchronize(c.stream) != cudaSuccess) {
      rc = CC_ERR_CUDA;
      break;
    }
    // counts -> offsets (exclusive prefix sum); h[n] = number of triangles
    int64_t run = 0;
    for (int64_t u = 0; u < n; u++) {
      const int64_t t = h[u];
      h[u] = run;
      run += t;
    }
    h[n] = run;
    // the list stays within a quarter of the memory left to this context
    size_t room = 0;
    if (c.budget) {
      room = c.budget > c.in_use ? (c.budget - c.in_use) / 4 : 0;
    } else {
      size_t fr = 0, tot = 0;
      if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { rc = CC_ERR_CUDA; break; }
      room = fr / 4;
    }
    const size_t nt = (size_t)std::max<int64_t>(run, 1);
    if (nt * 36 > room) {
      g.tri_state = -1;
      break;
    }
    g.tri_u = (int32_t *)dev_alloc(c, nt * 4);
    g.tri_v = (int32_t *)dev_alloc(c, nt * 4);
    g.tri_w = (int32_t *)dev_alloc(c, nt * 4);
    g.tri_p = (int64_t *)dev_alloc(c, nt * 24);
    g.n_tri = run;
    g.tri_state = 1;
    if (!g.tri_u || !g.tri_v || !g.tri_w || !g.tri_p) {
      tri_list_free(c, g);
      g.tri_state = -1;
      break;
    }
    if (cudaMemcpyAsync(counts, h.data(), (size_t)n * 8, cudaMemcpyHostToDevice, c.stream) != cudaSuccess) {
      rc = CC_ERR_CUDA;
      break;
    }
    rc = tl_launch(c, gv, true, nullptr, counts, g.tri_u, g.tri_v, g.tri_w, g.tri_p, g.n_tri, work, max_slots, smem);
    if (rc == CC_OK && cudaStreamSynchronize(c.stream) != cudaSuccess) rc = CC_ERR_CUDA;
  } while (false);
  timing_end(c);
  if (rc != CC_OK) tri_list_free(c, g);
  cudaStreamSynchronize(c.stream);
  dev_free(c, counts, (size_t)(n + 1) * 8);
  dev_free(c, work, 256);
  return rc;
}

int prepare_plan_graph(Ctx &c, DevGraph &g, const Plan &p) {
  if (!c.tri_list || g.tri_state != 0 || !g.owned) return CC_OK;
  for (auto &st : p.stages)
    if (st.kind == ST_TRI) return tri_list_build(c, g);
  return CC_OK;
}

// Stream the triangle list for one colouring: a block takes tiles of
// consecutive triangles (grouped by their highest vertex u); contributions
// to the tile's first source's own row (or its root count) gather in shared
// memory and reach global memory once per tile, the rest go by atomics.
constexpr int kEmitThreads = 256;
constexpr int kEmitTile = 2048;

template <int kForm>
__global__ void __launch_bounds__(kEmitThreads) k_tl_emit(TriArgs a, TriMode md, int R_acc) {
  extern __shared__ __align__(16) unsigned char emit_smem[];
  u64 *acc = reinterpret_cast<u64 *>(emit_smem);
  __shared__ u64 s_root;
  __shared__ int32_t s_u0;
  const int tid = threadIdx.x;
  unsigned ovf = 0;
  u64 other = 0;  // root counts of triangles whose source is not the tile's first
  for (int i = tid; i < R_acc; i += blockDim.x) acc[i] = 0;
  if (tid == 0) s_root = 0;
  for (int64_t t0 = (int64_t)blockIdx.x * kEmitTile; t0 < a.n_tri; t0 += (int64_t)gridDim.x * kEmitTile) {
    if (tid == 0) s_u0 = __ldg(a.tri_u + t0);
    __syncthreads();
    const int32_t u0 = s_u0;
    USink sk;
    if (a.nb == 1) sk.u = u0, sk.acc = acc;
    const int64_t t1 = min(a.n_tri, t0 + kEmitTile);
    for (int64_t i = t0 + tid; i < t1; i += blockDim.x) {
      const int32_t u = __ldg(a.tri_u + i), v = __ldg(a.tri_v + i), w = __ldg(a.tri_w + i);
      if (!cc_in(u, a.g.n, a.status) || !cc_in(v, u, a.status) || !cc_in(w, v, a.status)) continue;
      const int cu = a.colors[u], cv = a.colors[v], cw = a.colors[w];
      if (cu == cv || cu == cw || cv == cw) continue;
      u64 r = 0;
      const int64_t p01 = md.need_pos ? __ldg(a.tri_p + i) : 0;
      const int64_t p02 = md.need_pos ? __ldg(a.tri_p + a.n_tri + i) : 0;
      const int64_t p12 = md.need_pos ? __ldg(a.tri_p + 2 * a.n_tri + i) : 0;
      if (!cc_in(p01, a.g.nnz, a.status) || !cc_in(p02, a.g.nnz, a.status) || !cc_in(p12, a.g.nnz, a.status))
        continue;
      tri_visit<kForm>(a, md, sk, u, v, w, cu, cv, cw, p01, p02, p12, r, ovf);
      if (a.nb == 0 && r) {
        if (u == u0) {
          atomic_add_ck(&s_root, r, ovf);
        } else {
          other = add_ck(other, r, ovf);
          if (a.per_vertex) atomicAdd(a.per_vertex + u, r);
        }
      }
    }
    __syncthreads();
    if (a.nb == 1) {
      for (int k = tid; k < R_acc; k += blockDim.x) {
        const u64 t = acc[k];
        if (t) {
          atomic_add_ck(a.out + (int64_t)u0 * a.R_out + k, t, ovf);
          acc[k] = 0;
        }
      }
    }
    if (a.nb == 0 && tid == 0) {
      const u64 r = s_root;
      if (r) {
        atomic_add_ck(a.status + ST_COUNT, r, ovf);
        if (a.per_vertex) atomicAdd(a.per_vertex + u0, r);
      }
      s_root = 0;
    }
  }
  if (a.nb == 0) {
    other = warp_sum_ck(other, ovf);
    if ((tid & 31) == 0 && other) atomic_add_ck(a.status + ST_COUNT, other, ovf);
  }
  flag_overflow(a.status, ovf & 1u);
  if (ovf & 2u) atomicOr(a.status + ST_TIMEOUT, 2ull);  // partial list capacity exceeded
}

template <int kForm>
static int launch_emit(Ctx &c, const TriArgs &a, const TriMode &md, const char *name) {
  const int R_acc = a.nb == 1 ? ((a.R_out + 1) & ~1) : 0;
  const size_t smem = (size_t)std::max(R_acc, 2) * 8;
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(k_tl_emit<kForm>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return CC_ERR_CUDA;
  if (a.n_tri == 0) return CC_OK;
  const int64_t tiles = (a.n_tri + kEmitTile - 1) / kEmitTile;
  const int grid = (int)std::min<int64_t>(tiles, 152 * 8);
  timing_begin(c, name);
  k_tl_emit<kForm><<<grid, kEmitThreads, smem, c.stream>>>(a, md, R_acc);
  c.kernels++;
  timing_end(c);
  return cudaGetLastError() == cudaSuccess ? CC_OK : CC_ERR_CUDA;
}

template <int kForm>
int launch_triangle_form(Ctx &c, const TriArgs &a, const TriMode &md, const char *name) {
  // sources of degree >= kHubDegree: ranks [u_lo, n) (degree grows with rank)
  const int64_t n = a.g.n;
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) / 2;
    if (c.cur_graph_row[mid + 1] - c.cur_graph_row[mid] >= kHubDegree) hi = mid;
    else lo = mid + 1;
  }
  const int32_t u_lo = (int32_t)lo;
  int max_slots = 64, R_acc = 0;
  size_t smem = 0;
  int64_t grid = 0;
  if (u_lo < n) {
    const int64_t max_deg = c.cur_graph_row[n] - c.cur_graph_row[n - 1];
    while (max_slots < kHubMaxSlots && max_slots < 2 * max_deg) max_slots <<= 1;
    R_acc = a.nb == 1 ? ((a.R_out + 1) & ~1) : 0;
    smem = (size_t)R_acc * 8 + (size_t)max_slots * (md.need_pos ? 6 : 4);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_triangle_hub<kForm>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return CC_ERR_CUDA;
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_triangle_hub<kForm>, kHubThreads, smem) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device) != cudaSuccess)
      return CC_ERR_CUDA;
    grid = std::min<int64_t>((int64_t)std::max(per_sm, 1) * sms, n - u_lo);
  }
  int rc = CC_OK;
  timing_begin(c, name);
  if (u_lo < n) {
    if (cudaMemsetAsync(a.work_counter, 0, sizeof(int), c.stream) != cudaSuccess) {
      rc = CC_ERR_CUDA;
    } else {
      k_triangle_hub<kForm><<<(int)grid, kHubThreads, smem, c.stream>>>(a, md, u_lo, max_slots, R_acc);
      c.kernels++;
      if (cudaGetLastError() != cudaSuccess) rc = CC_ERR_CUDA;
    }
  }
  if (rc == CC_OK && u_lo > 0) {
    if (cudaMemsetAsync(a.work_counter, 0, sizeof(int), c.stream) != cudaSuccess) {
      rc = CC_ERR_CUDA;
    } else {
      k_triangle<kForm><<<152 * 8, 256, 0, c.stream>>>(a, md, u_lo);
      c.kernels++;
      if (cudaGetLastError() != cudaSuccess) rc = CC_ERR_CUDA;
    }
  }
  timing_end(c);
  return rc;
}

int launch_triangle(Ctx &c, const TriArgs &a_in) {
  TriArgs a = a_in;
  const DevGraph *g = c.cur_graph;
  // the triangle list when the graph has one (the structural counting pass
  // scans the wedges, which is the work it counts)
  const bool listed = c.tri_list && !a.count_units && g && g->tri_state == 1;
  if (listed) {
    a.n_tri = g->n_tri;
    a.tri_u = g->tri_u;
    a.tri_v = g->tri_v;
    a.tri_w = g->tri_w;
    a.tri_p = g->tri_p;
  }
  TriMode md;
  int n_ann = 0;
  bool any_edge = false;
  for (int i = 0; i < 3; i++) {
    md.plain = md.plain && !a.N[i].p && !a.E[i].p;
    if (a.N[i].p) n_ann++, md.one_pos = i, md.one_edge = false;
    if (a.E[i].p) n_ann++, md.one_pos = i, md.one_edge = true, any_edge = true;
  }
  if (n_ann != 1) md.one_pos = -1;
  md.need_pos = any_edge || a.nb == 2;
  if (listed) {
    if (md.plain) return launch_emit<0>(c, a, md, "triangle_list_plain");
    if (md.one_pos >= 0) return launch_emit<1>(c, a, md, "triangle_list_join1");
    return launch_emit<2>(c, a, md, "triangle_list_join");
  }
  if (md.plain) return launch_triangle_form<0>(c, a, md, "triangle_plain");
  if (md.one_pos >= 0) return launch_triangle_form<1>(c, a, md, "triangle_join1");
  return launch_triangle_form<2>(c, a, md, "triangle_join");
}

}  // namespace cc
