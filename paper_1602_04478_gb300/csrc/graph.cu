// Data-graph set-up on the device and the colouring kernel.
//
// K0 (degree order, Section 5.1): vertices are ordered by (degree, caller id)
// ascending and renamed by their rank, so "u is higher than w" becomes
// u > w.  The CSR is rebuilt in rank ids with every row sorted, which puts
// each vertex's lower neighbours in a row prefix (lo_cnt) and lets a source
// u find N(v) restricted to ranks below u by one binary search.  rev[e]
// gives the position of the reverse directed edge (edge-keyed tables store
// one row per directed edge; the transpose of Section 5.2 is a rev lookup).
// The same pass checks the graph: symmetric, no self-loops, no duplicates.
//
// K1 (colouring, Section 2): colour of caller id v in trial t is
// hi64(mix(seed ^ G(t+1) ^ mix(v)) * k), written in rank order.
#include <cub/cub.cuh>

#include <algorithm>
#include <vector>

#include "cc_device.cuh"
#include "cc_internal.h"
#include "cc_kernels.h"

namespace cc {

#define CK(x)                                   \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) return CC_ERR_CUDA;  \
  } while (0)

__device__ __forceinline__ unsigned long long sm64_mix(unsigned long long x) {
  unsigned long long z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Sort keys pack (major << bn) | minor, bn = the bits of a vertex id, so the
// radix sorts cover only the bits in use.
__global__ void k_degree_keys(int64_t n, const int64_t *row_ptr, unsigned long long *keys, int bn) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v < n) keys[v] = ((unsigned long long)(row_ptr[v + 1] - row_ptr[v]) << bn) | (unsigned long long)v;
}

__global__ void k_rank_of(int64_t n, const unsigned long long *sorted, int32_t *id_of, int32_t *rank_of, int bn) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r < n) {
    int32_t v = (int32_t)(sorted[r] & ((1ull << bn) - 1ull));
    id_of[r] = v;
    rank_of[v] = (int32_t)r;
  }
}

// one warp per original row: edge keys (rank(src) << bn | rank(dst)); also
// flags ids out of range
__global__ void k_edge_keys(int64_t n, const int64_t *row_ptr, const int32_t *col, const int32_t *rank_of,
                            unsigned long long *keys, unsigned long long *status, int bn) {
  int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= n) return;
  unsigned long long rs = (unsigned long long)rank_of[warp] << bn;
  for (int64_t e = row_ptr[warp] + lane; e < row_ptr[warp + 1]; e += 32) {
    int32_t c = col[e];
    if (c < 0 || c >= n) {
      atomicOr(status + ST_BADGRAPH, 1ull);
      keys[e] = rs;
      continue;
    }
    keys[e] = rs | (unsigned long long)(uint32_t)rank_of[c];
  }
}

__global__ void k_split_keys(int64_t nnz, const unsigned long long *keys, int32_t *col, int bn) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < nnz) col[e] = (int32_t)(keys[e] & ((1ull << bn) - 1ull));
}

static int bits_for(unsigned long long x) {
  int b = 1;
  while (b < 63 && (x >> b) != 0ull) b++;
  return b;
}

// warp per (rank-ordered) row: validity, lower-neighbour count, reverse edges
__global__ void k_finish_rows(int64_t n, const int64_t *row, const int32_t *col, int64_t *rev,
                              int32_t *lo_cnt, unsigned long long *status) {
  int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (r >= n) return;
  int64_t b = row[r], e = row[r + 1];
  if (lane == 0) lo_cnt[r] = (int32_t)(lower_bound_i32(col, b, e, (int32_t)r) - b);
  for (int64_t i = b + lane; i < e; i += 32) {
    int32_t c = col[i];
    bool bad = (c == (int32_t)r) || (i > b && col[i - 1] == c);
    int64_t p = lower_bound_i32(col, row[c], row[c + 1], (int32_t)r);
    if (p >= row[c + 1] || col[p] != (int32_t)r) bad = true;
    rev[i] = bad ? i : p;
    if (bad) atomicOr(status + ST_BADGRAPH, 1ull);
  }
}

__global__ void k_colors(int64_t n, const int32_t *id_of, unsigned long long seed, long long trial, int k,
                         uint8_t *out) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n) return;
  unsigned long long v = (unsigned long long)(uint32_t)id_of[r];
  unsigned long long h = sm64_mix(seed ^ (0x9E3779B97F4A7C15ull * (unsigned long long)(trial + 1)) ^ sm64_mix(v));
  out[r] = (uint8_t)__umul64hi(h, (unsigned long long)k);
}

__global__ void k_permute_colors(int64_t n, const int32_t *id_of, const uint8_t *by_id, uint8_t *by_rank) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r < n) by_rank[r] = by_id[id_of[r]];
}

static inline unsigned blocks_for(int64_t items, int per) { return (unsigned)((items + per - 1) / per); }

void graph_free(Ctx &c, DevGraph &g) {
  if (g.colors) dev_free(c, g.colors, (size_t)g.colors_T * g.n);
  g.colors = nullptr;
  tri_list_free(c, g);  // frees only what this context owns
  if (!g.owned) {  // a shared graph: its arrays belong to the context that loaded it
    g = DevGraph();
    return;
  }
  dev_free(c, g.row, (g.n + 1) * sizeof(int64_t));
  dev_free(c, g.col, std::max<int64_t>(g.nnz, 1) * sizeof(int32_t));
  dev_free(c, g.rev, std::max<int64_t>(g.nnz, 1) * sizeof(int64_t));
  dev_free(c, g.lo_cnt, g.n * sizeof(int32_t));
  dev_free(c, g.id_of, g.n * sizeof(int32_t));
  dev_free(c, g.rank_of, g.n * sizeof(int32_t));
  g = DevGraph();
}

int graph_load(Ctx &c, int64_t n, const int64_t *row_ptr, const int32_t *col, int64_t nnz, DevGraph &g) {
  if (n <= 0 || n >= (int64_t)1 << 31 || nnz < 0 || !row_ptr || (nnz > 0 && !col)) return CC_ERR_INVALID_ARG;
  if (row_ptr[0] != 0 || row_ptr[n] != nnz) return CC_ERR_BAD_GRAPH;
  int64_t deg_max = 0;
  for (int64_t v = 0; v < n; v++) {
    if (row_ptr[v + 1] < row_ptr[v]) return CC_ERR_BAD_GRAPH;
    deg_max = std::max<int64_t>(deg_max, row_ptr[v + 1] - row_ptr[v]);
  }
  // key widths: vertex ids (and ranks) below 2^bn, degrees below 2^bd
  const int bn = bits_for((unsigned long long)(n - 1)), bd = bits_for((unsigned long long)deg_max);
  cudaStream_t st = c.stream;
  g = DevGraph();
  g.n = n;
  g.nnz = nnz;
  int64_t nz1 = std::max<int64_t>(nnz, 1);
  g.row = (int64_t *)dev_alloc(c, (n + 1) * sizeof(int64_t));
  g.col = (int32_t *)dev_alloc(c, nz1 * sizeof(int32_t));
  g.rev = (int64_t *)dev_alloc(c, nz1 * sizeof(int64_t));
  g.lo_cnt = (int32_t *)dev_alloc(c, n * sizeof(int32_t));
  g.id_of = (int32_t *)dev_alloc(c, n * sizeof(int32_t));
  g.rank_of = (int32_t *)dev_alloc(c, n * sizeof(int32_t));
  if (!g.row || !g.col || !g.rev || !g.lo_cnt || !g.id_of || !g.rank_of) {
    graph_free(c, g);
    return CC_ERR_OOM;
  }
  // temporaries: original CSR, sort keys, CUB workspace
  int64_t *d_rp = (int64_t *)dev_alloc(c, (n + 1) * sizeof(int64_t));
  int32_t *d_col = (int32_t *)dev_alloc(c, nz1 * sizeof(int32_t));
  unsigned long long *k0 = (unsigned long long *)dev_alloc(c, std::max(n, nz1) * 8);
  unsigned long long *k1 = (unsigned long long *)dev_alloc(c, std::max(n, nz1) * 8);
  size_t tb1 = 0, tb2 = 0;
  cub::DeviceRadixSort::SortKeys(nullptr, tb1, k0, k1, n, 0, 64, st);
  cub::DeviceRadixSort::SortKeys(nullptr, tb2, k0, k1, nz1, 0, 64, st);
  size_t tb = std::max(tb1, tb2);
  void *tmp = dev_alloc(c, tb);
  int rc = CC_OK;
  auto cleanup = [&]() {
    dev_free(c, d_rp, (n + 1) * sizeof(int64_t));
    dev_free(c, d_col, nz1 * sizeof(int32_t));
    dev_free(c, k0, std::max(n, nz1) * 8);
    dev_free(c, k1, std::max(n, nz1) * 8);
    dev_free(c, tmp, tb);
  };
  if (!d_rp || !d_col || !k0 || !k1 || !tmp) {
    cleanup();
    graph_free(c, g);
    return CC_ERR_OOM;
  }
  do {
    if (cudaMemsetAsync(c.d_status, 0, 4 * sizeof(unsigned long long), st) != cudaSuccess) { rc = CC_ERR_CUDA; break; }
    if (cudaMemcpyAsync(d_rp, row_ptr, (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        (nnz > 0 && cudaMemcpyAsync(d_col, col, nnz * sizeof(int32_t), cudaMemcpyHostToDevice, st) != cudaSuccess)) {
      rc = CC_ERR_CUDA;
      break;
    }
    k_degree_keys<<<blocks_for(n, 256), 256, 0, st>>>(n, d_rp, k0, bn);
    c.kernels++;
    size_t tbx = tb;
    if (cub::DeviceRadixSort::SortKeys(tmp, tbx, k0, k1, n, 0, bn + bd, st) != cudaSuccess) { rc = CC_ERR_CUDA; break; }
    k_rank_of<<<blocks_for(n, 256), 256, 0, st>>>(n, k1, g.id_of, g.rank_of, bn);
    c.kernels++;
    // rank-ordered row pointers on the host (degrees are known there)
    std::vector<int32_t> id_of(n);
    if (cudaMemcpyAsync(id_of.data(), g.id_of, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rc = CC_ERR_CUDA;
      break;
    }
    g.h_row.assign(n + 1, 0);
    for (int64_t r = 0; r < n; r++) g.h_row[r + 1] = g.h_row[r] + (row_ptr[id_of[r] + 1] - row_ptr[id_of[r]]);
    g.max_deg = n > 0 ? g.h_row[n] - g.h_row[n - 1] : 0;
    if (cudaMemcpyAsync(g.row, g.h_row.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st) != cudaSuccess) {
      rc = CC_ERR_CUDA;
      break;
    }
    if (nnz > 0) {
      k_edge_keys<<<blocks_for(n * 32, 256), 256, 0, st>>>(n, d_rp, d_col, g.rank_of, k0, c.d_status, bn);
      c.kernels++;
      tbx = tb;
      if (cub::DeviceRadixSort::SortKeys(tmp, tbx, k0, k1, nnz, 0, 2 * bn, st) != cudaSuccess) { rc = CC_ERR_CUDA; break; }
      k_split_keys<<<blocks_for(nnz, 256), 256, 0, st>>>(nnz, k1, g.col, bn);
      c.kernels++;
    }
    k_finish_rows<<<blocks_for(n * 32, 256), 256, 0, st>>>(n, g.row, g.col, g.rev, g.lo_cnt, c.d_status);
    c.kernels++;
    unsigned long long status[4];
    if (cudaMemcpyAsync(status, c.d_status, sizeof(status), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rc = CC_ERR_CUDA;
      break;
    }
    if (status[ST_BADGRAPH]) rc = CC_ERR_BAD_GRAPH;
  } while (0);
  if (rc == CC_OK && cudaGetLastError() != cudaSuccess) rc = CC_ERR_CUDA;
  cleanup();
  if (rc != CC_OK) graph_free(c, g);
  return rc;
}

int colors_fill(Ctx &c, const DevGraph &g, int k, int64_t trial, uint8_t *d_out) {
  if (g.colors) {
    if (trial < 0 || trial >= g.colors_T) return CC_ERR_INVALID_ARG;
    cudaMemcpyAsync(d_out, g.colors + (size_t)trial * g.n, g.n, cudaMemcpyDeviceToDevice, c.stream);
  } else {
    k_colors<<<blocks_for(g.n, 256), 256, 0, c.stream>>>(g.n, g.id_of, c.seed, trial, k, d_out);
    c.kernels++;
  }
  return cudaGetLastError() == cudaSuccess ? CC_OK : CC_ERR_CUDA;
}

int colors_set(Ctx &c, DevGraph &g, const uint8_t *h_colors, int T) {
  if (g.colors) dev_free(c, g.colors, (size_t)g.colors_T * g.n);
  g.colors = nullptr;
  g.colors_T = 0;
  if (T <= 0) return CC_OK;
  uint8_t *d_by_id = (uint8_t *)dev_alloc(c, (size_t)g.n);
  uint8_t *d = (uint8_t *)dev_alloc(c, (size_t)T * g.n);
  if (!d_by_id || !d) {
    dev_free(c, d_by_id, g.n);
    dev_free(c, d, (size_t)T * g.n);
    return CC_ERR_OOM;
  }
  for (int t = 0; t < T; t++) {
    CK(cudaMemcpyAsync(d_by_id, h_colors + (size_t)t * g.n, g.n, cudaMemcpyHostToDevice, c.stream));
    k_permute_colors<<<blocks_for(g.n, 256), 256, 0, c.stream>>>(g.n, g.id_of, d_by_id, d + (size_t)t * g.n);
    c.kernels++;
  }
  CK(cudaStreamSynchronize(c.stream));
  dev_free(c, d_by_id, g.n);
  g.colors = d;
  g.colors_T = T;
  return CC_OK;
}

// colex rank / unrank tables for masks of up to 12 bits
int luts_init(Ctx &c) {
  std::vector<uint16_t> rank(4096, 0), unrank(13 * kUnrankStride, 0);
  int binom[13][13] = {{0}};
  for (int a = 0; a <= 12; a++) {
    binom[a][0] = 1;
    for (int b = 1; b <= a; b++) binom[a][b] = binom[a - 1][b - 1] + (b <= a - 1 ? binom[a - 1][b] : 0);
  }
  for (uint32_t m = 0; m < 4096; m++) {
    int r = 0, i = 0;
    for (int p = 0; p < 12; p++)
      if (m >> p & 1) {
        i++;
        r += (i <= p) ? binom[p][i] : 0;
      }
    rank[m] = (uint16_t)r;
    unrank[__builtin_popcount(m) * kUnrankStride + r] = (uint16_t)m;
  }
  c.lut_rank = (uint16_t *)dev_alloc(c, rank.size() * 2);
  c.lut_unrank = (uint16_t *)dev_alloc(c, unrank.size() * 2);
  if (!c.lut_rank || !c.lut_unrank) return CC_ERR_OOM;
  CK(cudaMemcpyAsync(c.lut_rank, rank.data(), rank.size() * 2, cudaMemcpyHostToDevice, c.stream));
  CK(cudaMemcpyAsync(c.lut_unrank, unrank.data(), unrank.size() * 2, cudaMemcpyHostToDevice, c.stream));
  CK(cudaStreamSynchronize(c.stream));
  return CC_OK;
}

}  // namespace cc
