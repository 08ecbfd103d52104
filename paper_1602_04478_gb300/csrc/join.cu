// K2: leaf-block join and K6: root-singleton reduction.
//
// Leaf block (a, b) with b a leaf (Section 5.2, "leaf blocks"): join the
// tables of the blocks annotating node a, edge (a, b) and node b.  For a data
// vertex x as the image of a:
//   Y[x][S]   = sum over neighbours y of x of  E[(x,y)][S_E] * B[y][S_B]
//               with S_E containing chi(x), chi(y), S_B containing chi(y),
//               S_E and S_B sharing exactly chi(y), S = S_E u S_B;
//   Out[x][S] = sum over S_A, S_Y with S_A and S_Y sharing exactly chi(x),
//               S = S_A u S_Y, of A[x][S_A] * Y[x][S_Y].
// A missing block is the identity (A: the single signature {chi(x)}; B:
// {chi(y)}; E: the plain data edge with signature {chi(x), chi(y)}, count 1
// when the two colours differ -- the B_G table of Section 5.2).
// One warp per vertex; Y lives in shared memory.  The gather of B rows over
// the CSR is the HBM traffic of this kernel.
//
// Root singleton (Section 5.2, last paragraph): sum the annotating block's
// table over all vertices (its rows hold the single full signature).
#include <algorithm>

#include "cc_kernels.h"

namespace cc {

__global__ void __launch_bounds__(256) k_leaf_join(LeafArgs a) {
  extern __shared__ u64 smem_y[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  u64 *Y = smem_y + (size_t)wib * a.RY;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  unsigned ovf = 0;
  for (int64_t x = blockIdx.x * (int64_t)(blockDim.x >> 5) + wib; x < a.g.n; x += nwarps) {
    const int cx = a.colors[x];
    for (int i = lane; i < a.RY; i += 32) Y[i] = 0;
    __syncwarp();
    const int64_t rb = a.g.row[x], re = a.g.row[x + 1];
    for (int64_t i = rb + lane; i < re; i += 32) {
      const int32_t y = __ldg(a.g.col + i);
      const int cy = a.colors[y];
      if (cy == cx) continue;
      const int nE = a.E.p ? a.E.R : 1;
      const int64_t erow = a.E.p ? (a.E.use_rev ? __ldg(a.g.rev + i) : i) : 0;
      for (int je = 0; je < nE; je++) {
        uint32_t mE;
        u64 vE;
        if (a.E.p) {
          vE = __ldg(a.E.p + erow * a.E.R + je);
          if (!vE) continue;
          mE = pmask(a.lut, a.E.s, je, cx, cy);
        } else {
          vE = 1;
          mE = (1u << cx) | (1u << cy);
        }
        if (a.B.p) {
          const u64 *brow = a.B.p + (int64_t)y * a.B.R;
          for (int jb = 0; jb < a.B.R; jb++) {
            u64 vB = __ldg(brow + jb);
            if (!vB) continue;
            uint32_t mB = umask(a.lut, a.B.s, jb, cy);
            if ((mB & mE) != (1u << cy)) continue;
            u64 v = mul_ck(vE, vB, ovf);
            int slot = uslot(a.lut, mB | mE, cx);
            unsigned long long old = atomicAdd(Y + slot, v);
            ovf |= (old + v < old);
          }
        } else {
          int slot = uslot(a.lut, mE, cx);
          unsigned long long old = atomicAdd(Y + slot, vE);
          ovf |= (old + vE < old);
        }
      }
    }
    __syncwarp();
    u64 *orow = a.out + x * (int64_t)a.R_out;
    if (!a.A.p) {
      for (int o = lane; o < a.R_out; o += 32) orow[o] = Y[o];
    } else {
      const u64 *arow = a.A.p + x * (int64_t)a.A.R;
      for (int o = lane; o < a.R_out; o += 32) {
        uint32_t mO = umask(a.lut, a.s_out, o, cx);
        u64 acc = 0;
        for (int ja = 0; ja < a.A.R; ja++) {
          u64 vA = __ldg(arow + ja);
          if (!vA) continue;
          uint32_t mA = umask(a.lut, a.A.s, ja, cx);
          if (mA & ~mO) continue;
          uint32_t mY = (mO & ~mA) | (1u << cx);
          u64 vY = Y[uslot(a.lut, mY, cx)];
          if (!vY) continue;
          acc = add_ck(acc, mul_ck(vA, vY, ovf), ovf);
        }
        orow[o] = acc;
      }
    }
    __syncwarp();
  }
  flag_overflow(a.status, ovf);
}

// The same join for a leaf block with no edge table (the edge is a plain data
// edge), one warp per vertex x with the lanes over the (neighbour, B-row
// entry) pairs of x: consecutive lanes read consecutive entries of a
// neighbour's row, so the gather is coalesced, and the signature arithmetic
// is one lookup in a table built per block in shared memory:
//   slot[(cx k + cy) RB + j] = the slot of S_B(j) u {cx} in x's Y row, or -1
//   when S_B(j) holds cx (the signatures would overlap beyond chi(y)).
// Without a B table the neighbour's row is the single signature {cy}.
constexpr int kFlatMaxTable = 8192;

__global__ void __launch_bounds__(256) k_leaf_join_flat(LeafArgs a) {
  extern __shared__ __align__(16) unsigned char flat_smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int k = a.k;
  const int RB = a.B.p ? a.B.R : 1;
  const int sB = a.B.p ? a.B.s : 1;
  u64 *Y = reinterpret_cast<u64 *>(flat_smem) + (size_t)wib * a.RY;
  int16_t *tbl = reinterpret_cast<int16_t *>(reinterpret_cast<u64 *>(flat_smem) + (size_t)8 * a.RY);
  for (int t = threadIdx.x; t < k * k * RB; t += blockDim.x) {
    const int j = t % RB, cy = (t / RB) % k, cx = t / (RB * k);
    const uint32_t mB = a.B.p ? umask(a.lut, sB, j, cy) : (1u << cy);
    tbl[t] = (cx == cy || (mB >> cx & 1u)) ? (int16_t)-1 : (int16_t)uslot(a.lut, mB | (1u << cx), cx);
  }
  __syncthreads();
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  // this lane's starting (neighbour, entry) pair and its step per pass
  const int i0 = lane / RB, j0 = lane % RB, di = 32 / RB, dj = 32 % RB;
  unsigned ovf = 0;
  for (int64_t x = blockIdx.x * (int64_t)(blockDim.x >> 5) + wib; x < a.g.n; x += nwarps) {
    const int cx = a.colors[x];
    for (int i = lane; i < a.RY; i += 32) Y[i] = 0;
    __syncwarp();
    const int64_t rb = a.g.row[x];
    const int deg = (int)(a.g.row[x + 1] - rb);
    const int16_t *tx = tbl + (size_t)cx * k * RB;
    for (int i = i0, j = j0; i < deg;) {
      const int32_t y = __ldg(a.g.col + rb + i);
      const bool ok = cc_in(y, a.g.n, a.status);
      const int cy = ok ? a.colors[y] : 0;
      const u64 v = !ok ? 0ull : (a.B.p ? __ldg(a.B.p + (int64_t)y * RB + j) : 1ull);
      const int slot = tx[cy * RB + j];
      // slot -1: the signatures overlap beyond chi(y), no match
      if (v && slot >= 0 && cc_in(slot, a.RY, a.status)) {
        const unsigned long long old = atomicAdd(Y + slot, v);
        ovf |= (old + v < old);
      }
      i += di;
      j += dj;
      if (j >= RB) j -= RB, i++;
    }
    __syncwarp();
    u64 *orow = a.out + x * (int64_t)a.R_out;
    if (!a.A.p) {
      for (int o = lane; o < a.R_out; o += 32) orow[o] = Y[o];
    } else {
      const u64 *arow = a.A.p + x * (int64_t)a.A.R;
      for (int o = lane; o < a.R_out; o += 32) {
        uint32_t mO = umask(a.lut, a.s_out, o, cx);
        u64 acc = 0;
        for (int ja = 0; ja < a.A.R; ja++) {
          u64 vA = __ldg(arow + ja);
          if (!vA) continue;
          uint32_t mA = umask(a.lut, a.A.s, ja, cx);
          if (mA & ~mO) continue;
          uint32_t mY = (mO & ~mA) | (1u << cx);
          u64 vY = Y[uslot(a.lut, mY, cx)];
          if (!vY) continue;
          acc = add_ck(acc, mul_ck(vA, vY, ovf), ovf);
        }
        orow[o] = acc;
      }
    }
    __syncwarp();
  }
  flag_overflow(a.status, ovf);
}

// The same join with the lanes on the output slots of Y (Y rows of at most
// 16 or 32 slots, no A and no edge table): for each neighbour y of x, lane s
// reads the one entry of y's row whose signature, with chi(x) added, is Y's
// slot s -- inv[(cx k + cy) RY + s], or -1 when there is none -- and adds it
// to its own register.  No atomics; a row's entries are read by neighbouring
// lanes.  With Y rows of at most 16 slots each half-warp takes its own
// neighbours and the halves are summed at the end.  Neighbour ids and their
// colours are read 32 at a time (one per lane) and passed round by shuffles,
// and four neighbours' row entries are loaded before any is added, so each
// lane has four independent gathers in flight instead of a chain of three
// dependent loads per neighbour.
__global__ void __launch_bounds__(256) k_leaf_join_slots(LeafArgs a) {
  extern __shared__ __align__(16) unsigned char slots_smem[];
  int16_t *inv = reinterpret_cast<int16_t *>(slots_smem);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int k = a.k, RY = a.RY;
  const int RB = a.B.p ? a.B.R : 1;
  const int sB = a.B.p ? a.B.s : 1;
  for (int t = threadIdx.x; t < k * k * RY; t += blockDim.x) inv[t] = -1;
  __syncthreads();
  for (int t = threadIdx.x; t < k * k * RB; t += blockDim.x) {
    const int j = t % RB, cy = (t / RB) % k, cx = t / (RB * k);
    const uint32_t mB = a.B.p ? umask(a.lut, sB, j, cy) : (1u << cy);
    if (cx != cy && !(mB >> cx & 1u)) inv[(cx * k + cy) * RY + uslot(a.lut, mB | (1u << cx), cx)] = (int16_t)j;
  }
  __syncthreads();
  const bool halves = RY <= 16;
  const int s = halves ? (lane & 15) : lane;  // this lane's output slot
  const int h = halves ? (lane >> 4) : 0;     // which neighbours: h, h + step, ...
  const int step = halves ? 2 : 1;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  unsigned ovf = 0;
  for (int64_t x = blockIdx.x * (int64_t)(blockDim.x >> 5) + wib; x < a.g.n; x += nwarps) {
    const int cx = a.colors[x];
    const int64_t rb = a.g.row[x];
    const int deg = (int)(a.g.row[x + 1] - rb);
    const int16_t *ix = inv + (size_t)cx * k * RY;
    u64 acc = 0;
    for (int base = 0; base < deg; base += 32) {
      // this chunk's neighbours and colours, one per lane
      const int cnt = min(32, deg - base);
      int32_t yl = lane < cnt ? __ldg(a.g.col + rb + base + lane) : -1;
      if (yl >= 0 && !cc_in(yl, a.g.n, a.status)) yl = -1;
      const int cl = yl >= 0 ? (int)a.colors[yl] : 0;
      for (int t0 = 0; t0 < cnt; t0 += 4 * step) {
        u64 v[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const int t = t0 + h + q * step;  // the neighbour this lane takes
          const int32_t y = __shfl_sync(0xffffffffu, yl, t & 31);
          const int cy = __shfl_sync(0xffffffffu, cl, t & 31);
          const int j = (t < cnt && s < RY && y >= 0) ? ix[cy * RY + s] : -1;
          v[q] = j < 0 ? 0ull : (a.B.p ? __ldg(a.B.p + (int64_t)y * RB + j) : 1ull);
        }
#pragma unroll
        for (int q = 0; q < 4; q++) acc = add_ck(acc, v[q], ovf);
      }
    }
    if (halves) acc = add_ck(acc, __shfl_down_sync(0xffffffffu, acc, 16), ovf);
    if (lane < RY) a.out[x * (int64_t)a.R_out + lane] = acc;
  }
  flag_overflow(a.status, ovf);
}

int launch_leaf(Ctx &c, const LeafArgs &a) {
  const int RB = a.B.p ? a.B.R : 1;
  if (!a.E.p && !a.A.p && a.RY <= 32 && a.RY == a.R_out && a.k * a.k * (a.RY + RB) <= kFlatMaxTable) {
    const size_t smem = (size_t)a.k * a.k * a.RY * sizeof(int16_t);
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(k_leaf_join_slots, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int64_t blocks = std::min<int64_t>(std::max<int64_t>((a.g.n + 7) / 8, 1), 152 * 8);
    timing_begin(c, "leaf_join");
    k_leaf_join_slots<<<(unsigned)blocks, 256, smem, c.stream>>>(a);
    c.kernels++;
    timing_end(c);
    return cudaGetLastError() == cudaSuccess ? CC_OK : CC_ERR_CUDA;
  }
  if (!a.E.p && a.k * a.k * RB <= kFlatMaxTable) {
    const size_t smem = (size_t)8 * a.RY * sizeof(u64) + (size_t)a.k * a.k * RB * sizeof(int16_t);
    if (smem > 200 * 1024) return CC_ERR_UNSUPPORTED;
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(k_leaf_join_flat, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int64_t blocks = std::min<int64_t>(std::max<int64_t>((a.g.n + 7) / 8, 1), 152 * 8);
    timing_begin(c, "leaf_join");
    k_leaf_join_flat<<<(unsigned)blocks, 256, smem, c.stream>>>(a);
    c.kernels++;
    timing_end(c);
    return cudaGetLastError() == cudaSuccess ? CC_OK : CC_ERR_CUDA;
  }
  size_t smem = (size_t)8 * a.RY * sizeof(u64);
  if (smem > 200 * 1024) return CC_ERR_UNSUPPORTED;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_leaf_join, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int64_t blocks = (a.g.n + 7) / 8;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  timing_begin(c, "leaf_join");
  k_leaf_join<<<(unsigned)blocks, 256, smem, c.stream>>>(a);
  c.kernels++;
  timing_end(c);
  return cudaGetLastError() == cudaSuccess ? CC_OK : CC_ERR_CUDA;
}

__global__ void __launch_bounds__(256) k_root_sum(int64_t n, const u64 *table, u64 *per_vertex, u64 *status) {
  unsigned ovf = 0;
  u64 acc = 0;
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
    u64 v = table[x];
    if (per_vertex) per_vertex[x] = v;
    acc = add_ck(acc, v, ovf);
  }
  acc = warp_sum_ck(acc, ovf);
  if ((threadIdx.x & 31) == 0) atomic_add_ck(status + ST_COUNT, acc, ovf);
  flag_overflow(status, ovf);
}

int launch_root_sum(Ctx &c, const GraphView &g, const u64 *table, u64 *per_vertex, u64 *status) {
  int64_t blocks = (g.n + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  timing_begin(c, "root_sum");
  k_root_sum<<<(unsigned)blocks, 256, 0, c.stream>>>(g.n, table, per_vertex, status);
  c.kernels++;
  timing_end(c);
  return cudaGetLastError() == cudaSuccess ? CC_OK : CC_ERR_CUDA;
}

}  // namespace cc
