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
// One warp per source u, sources taken highest first from a work counter.
#include "cc_kernels.h"

namespace cc {

constexpr int kMaxPartial = 128;

struct TriEdges {
  int64_t pos[3][3];  // pos[i][j]: CSR position of directed edge p_i -> p_j (local ids 0=u,1=v,2=w)
};

__device__ void tri_emit_plain(const TriArgs &a, const int32_t vx[3], const int c[3], const TriEdges &te,
                               u64 &root_acc, unsigned &ovf) {
  uint32_t S = (1u << c[0]) | (1u << c[1]) | (1u << c[2]);
  if (a.nb == 0) {
    root_acc = add_ck(root_acc, 6ull, ovf);
  } else if (a.nb == 1) {
    for (int i = 0; i < 3; i++)
      atomic_add_ck(a.out + (int64_t)vx[i] * a.R_out + uslot(a.lut, S, c[i]), 2ull, ovf);
  } else {
    for (int i = 0; i < 3; i++)
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

__device__ void tri_emit_general(const TriArgs &a, const int32_t vx[3], const int c[3], const TriEdges &te,
                                 u64 &root_acc, unsigned &ovf) {
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
        atomic_add_ck(a.out + (int64_t)vx[lb] * a.R_out + uslot(a.lut, pm[q], c[lb]), pv[q], ovf);
      } else {
        int l0 = p[a.bd[0]], l1 = p[a.bd[1]];
        atomic_add_ck(a.out + te.pos[l0][l1] * a.R_out + pslot(a.lut, pm[q], c[l0], c[l1]), pv[q], ovf);
      }
    }
  }
}

// One annotation only (a node table at position ai, or an edge table on edge
// ai -> ai+1): each of its row's signatures extends the triangle's colours
// directly, without partial lists.
__device__ __forceinline__ void tri_emit_one(const TriArgs &a, const int32_t vx[3], const int c[3],
                                             const TriEdges &te, u64 &root_acc, unsigned &ovf, int ai, bool edge) {
  const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  const uint32_t K = (1u << a.k) - 1u;
  for (int pi = 0; pi < 6; pi++) {
    const int *p = perms[pi];
    const uint32_t base = (1u << c[p[0]]) | (1u << c[p[1]]) | (1u << c[p[2]]);
    const int li = p[ai], lj = p[(ai + 1) % 3];
    const u64 *row;
    int R, s;
    uint32_t shared;
    if (edge) {
      const TabE &E = a.E[ai];
      int64_t e = E.use_rev ? te.pos[lj][li] : te.pos[li][lj];
      row = E.p + e * E.R;
      R = E.R;
      s = E.s;
      shared = (1u << c[li]) | (1u << c[lj]);
    } else {
      const TabU &N = a.N[ai];
      row = N.p + (int64_t)vx[li] * N.R;
      R = N.R;
      s = N.s;
      shared = 1u << c[li];
    }
    if (a.nb == 0) {
      // the root's signature is the full colour set: one compatible slot
      uint32_t m = (K & ~base) | shared;
      int slot = edge ? pslot(a.lut, m, c[li], c[lj]) : uslot(a.lut, m, c[li]);
      root_acc = add_ck(root_acc, __ldg(row + slot), ovf);
      continue;
    }
    for (int j = 0; j < R; j++) {
      u64 t = __ldg(row + j);
      if (!t) continue;
      uint32_t mt = edge ? pmask(a.lut, s, j, c[li], c[lj]) : umask(a.lut, s, j, c[li]);
      if ((mt & base) != shared) continue;
      uint32_t m = mt | base;
      if (a.nb == 1) {
        int lb = p[a.bd[0]];
        atomic_add_ck(a.out + (int64_t)vx[lb] * a.R_out + uslot(a.lut, m, c[lb]), t, ovf);
      } else {
        int l0 = p[a.bd[0]], l1 = p[a.bd[1]];
        atomic_add_ck(a.out + te.pos[l0][l1] * a.R_out + pslot(a.lut, m, c[l0], c[l1]), t, ovf);
      }
    }
  }
}

__global__ void __launch_bounds__(256) k_triangle(TriArgs a, bool plain, int one_pos, bool one_edge) {
  const int lane = threadIdx.x & 31;
  unsigned ovf = 0;
  while (true) {
    int idx = 0;
    if (lane == 0) idx = atomicAdd(a.work_counter, 1);
    idx = __shfl_sync(0xffffffffu, idx, 0);
    if (idx >= a.g.n) break;
    const int32_t u = (int32_t)(a.g.n - 1 - idx);
    const int64_t ub = a.g.row[u];
    const int du = a.g.lo_cnt[u];
    const int cu = a.colors[u];
    u64 root_acc = 0;
    u64 units = 0;
    for (int iv = 1; iv < du; iv++) {
      const int32_t v = __ldg(a.g.col + ub + iv);
      const int cv = a.colors[v];
      const int64_t vb = a.g.row[v];
      const int dv = a.g.lo_cnt[v];
      units += (u64)dv;
      for (int j = lane; j < dv; j += 32) {
        const int32_t w = __ldg(a.g.col + vb + j);
        // w must be a lower neighbour of u below v: search N<(u)[0, iv)
        int64_t p = lower_bound_i32(a.g.col, ub, ub + iv, w);
        if (p >= ub + iv || __ldg(a.g.col + p) != w) continue;
        const int cw = a.colors[w];
        // a colourful match maps the triangle to three distinct colours
        if (cu == cv || cu == cw || cv == cw) continue;
        int32_t vx[3] = {u, v, w};
        int c[3] = {cu, cv, cw};
        TriEdges te;
        te.pos[0][1] = ub + iv;
        te.pos[0][2] = p;
        te.pos[1][2] = vb + j;
        te.pos[1][0] = __ldg(a.g.rev + te.pos[0][1]);
        te.pos[2][0] = __ldg(a.g.rev + te.pos[0][2]);
        te.pos[2][1] = __ldg(a.g.rev + te.pos[1][2]);
        te.pos[0][0] = te.pos[1][1] = te.pos[2][2] = -1;
        if (plain) tri_emit_plain(a, vx, c, te, root_acc, ovf);
        else if (one_pos >= 0) tri_emit_one(a, vx, c, te, root_acc, ovf, one_pos, one_edge);
        else tri_emit_general(a, vx, c, te, root_acc, ovf);
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

int launch_triangle(Ctx &c, const TriArgs &a) {
  bool plain = true;
  int n_ann = 0, one_pos = -1;
  bool one_edge = false;
  for (int i = 0; i < 3; i++) {
    plain = plain && !a.N[i].p && !a.E[i].p;
    if (a.N[i].p) n_ann++, one_pos = i, one_edge = false;
    if (a.E[i].p) n_ann++, one_pos = i, one_edge = true;
  }
  if (n_ann != 1) one_pos = -1;
  if (cudaMemsetAsync(a.work_counter, 0, sizeof(int), c.stream) != cudaSuccess) return CC_ERR_CUDA;
  timing_begin(c, plain ? "triangle_plain" : (one_pos >= 0 ? "triangle_join1" : "triangle_join"));
  k_triangle<<<152 * 8, 256, 0, c.stream>>>(a, plain, one_pos, one_edge);
  timing_end(c);
  return cudaGetLastError() == cudaSuccess ? CC_OK : CC_ERR_CUDA;
}

}  // namespace cc
