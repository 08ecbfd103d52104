// Pair graphs of Case-2 blocks (Section 4.1, Case 2) whose boundary images
// need not be adjacent in the data graph.
//
// Such a block's projection table cnt(x, y, alpha | B) (Section 5, the
// binary projection tables) keeps only the nonzero (x, y) rows.  The cycle
// kernel appends them as a list of keys (x << 32 | y) with a row each; this
// file turns the list into a CSR over the data graph's vertices holding the
// symmetric closure of the keys, so that a parent cycle can walk the
// annotated edge in either direction exactly as it walks a data edge: rows
// ascending (the DB order test is a binary search), rev (the position of the
// reverse pair) and lo_cnt (the partners below the vertex).  Position q of a
// forward key keeps the index of its row; a position that exists only as the
// reverse of another key has no row (-1), and a walk over it reads zeros
// (its table row is read through rev, like a data edge traversed against the
// table's orientation).
#include <cub/cub.cuh>

#include <algorithm>

#include "cc_device.cuh"
#include "cc_internal.h"
#include "cc_kernels.h"

namespace cc {

namespace {

__global__ void k_pair_expand(const unsigned long long *keys, int64_t np, unsigned long long *k2, int64_t *v2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long key = keys[i];
    k2[i] = key;
    v2[i] = i;
    k2[np + i] = (key << 32) | (key >> 32);
    v2[np + i] = -1;
  }
}

// head[q] = 1 where a new key starts in the sorted list
__global__ void k_pair_heads(const unsigned long long *ks, int64_t m, int64_t *head) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m; q += (int64_t)gridDim.x * blockDim.x)
    head[q] = (q == 0 || ks[q] != ks[q - 1]) ? 1 : 0;
}

// one position per distinct key: partner, owner key, row index (a key
// appears at most twice: as itself and as the reverse of its partner's key)
__global__ void k_pair_scatter(const unsigned long long *ks, const int64_t *vs, const int64_t *pos, int64_t m,
                               int32_t *col, unsigned long long *ukeys, int64_t *ridx) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m; q += (int64_t)gridDim.x * blockDim.x) {
    if (q > 0 && ks[q] == ks[q - 1]) continue;
    const int64_t p = pos[q];
    col[p] = (int32_t)(uint32_t)(ks[q] & 0xffffffffull);
    ukeys[p] = ks[q];
    int64_t r = vs[q];
    if (r < 0 && q + 1 < m && ks[q + 1] == ks[q]) r = vs[q + 1];
    ridx[p] = r;
  }
}

__global__ void k_pair_rows(const unsigned long long *ukeys, int64_t nnz, int64_t n, int64_t *row) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v <= n; v += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long key = (unsigned long long)v << 32;
    int64_t lo = 0, hi = nnz;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (ukeys[mid] < key) lo = mid + 1;
      else hi = mid;
    }
    row[v] = lo;
  }
}

__global__ void k_pair_lo(const int64_t *row, const int32_t *col, int64_t n, int32_t *lo_cnt) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    lo_cnt[v] = (int32_t)(lower_bound_i32(col, row[v], row[v + 1], (int32_t)v) - row[v]);
}

__global__ void k_pair_rev(const unsigned long long *ukeys, const int64_t *row, const int32_t *col, int64_t nnz,
                           int64_t *rev) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = (int32_t)(ukeys[q] >> 32), x = col[q];
    rev[q] = lower_bound_i32(col, row[x], row[x + 1], u);
  }
}

// rows by position (the reverse-only positions zero) for kernels that index
// an edge-keyed table by CSR position
__global__ void k_pair_dense(const int64_t *ridx, const u64 *rows, int64_t nnz, int R, u64 *dense) {
  const int64_t total = nnz * R;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = i / R, r = ridx[q];
    dense[i] = r < 0 ? 0ull : rows[r * R + (i - q * R)];
  }
}

int grid_for(int64_t m) { return (int)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, 152 * 16)); }

}  // namespace

int pair_graph_sort(Ctx &c, int64_t n, const unsigned long long *keys, int64_t n_pairs, int64_t m, PairGraph &pg);

void pair_graph_free(Ctx &c, PairGraph &pg) {
  dev_free(c, pg.row, (size_t)(pg.n + 1) * 8);
  dev_free(c, pg.col, (size_t)std::max<int64_t>(pg.nnz, 1) * 4);
  dev_free(c, pg.rev, (size_t)std::max<int64_t>(pg.nnz, 1) * 8);
  dev_free(c, pg.lo_cnt, (size_t)std::max<int64_t>(pg.n, 1) * 4);
  dev_free(c, pg.ridx, (size_t)std::max<int64_t>(pg.nnz, 1) * 8);
  dev_free(c, pg.rows, (size_t)std::max<int64_t>(pg.rows_cap, 1) * pg.R * 8);
  pg = PairGraph();
}

// keys: the n_pairs distinct appended keys (device).  pg.rows, rows_cap and
// R are the caller's (the appended rows, kept as they are).  Synchronises.
int pair_graph_build(Ctx &c, int64_t n, const unsigned long long *keys, int64_t n_pairs, PairGraph &pg) {
  pg.n = n;
  pg.n_pairs = n_pairs;
  const int64_t m = 2 * n_pairs;
  cudaStream_t st = c.stream;
  pg.row = (int64_t *)dev_alloc(c, (size_t)(n + 1) * 8);
  pg.lo_cnt = (int32_t *)dev_alloc(c, (size_t)std::max<int64_t>(n, 1) * 4);
  if (!pg.row || !pg.lo_cnt) return CC_ERR_OOM;
  if (m == 0) {
    pg.nnz = 0;
    pg.col = (int32_t *)dev_alloc(c, 4);
    pg.rev = (int64_t *)dev_alloc(c, 8);
    pg.ridx = (int64_t *)dev_alloc(c, 8);
    if (!pg.col || !pg.rev || !pg.ridx) return CC_ERR_OOM;
    if (cudaMemsetAsync(pg.row, 0, (size_t)(n + 1) * 8, st) != cudaSuccess ||
        cudaMemsetAsync(pg.lo_cnt, 0, (size_t)std::max<int64_t>(n, 1) * 4, st) != cudaSuccess)
      return CC_ERR_CUDA;
    return CC_OK;
  }
  timing_begin(c, "pair_graph_build");
  const int rc_build = pair_graph_sort(c, n, keys, n_pairs, m, pg);
  timing_end(c);
  return rc_build;
}

int pair_graph_sort(Ctx &c, int64_t n, const unsigned long long *keys, int64_t n_pairs, int64_t m, PairGraph &pg) {
  cudaStream_t st = c.stream;
  size_t tb_sort = 0, tb_scan = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, tb_sort, (unsigned long long *)nullptr, (unsigned long long *)nullptr,
                                  (int64_t *)nullptr, (int64_t *)nullptr, (int)m, 0, 64, st);
  cub::DeviceScan::ExclusiveSum(nullptr, tb_scan, (int64_t *)nullptr, (int64_t *)nullptr, (int)m, st);
  const size_t tb = std::max(tb_sort, tb_scan);
  unsigned long long *k2 = (unsigned long long *)dev_alloc(c, (size_t)m * 8);
  unsigned long long *ks = (unsigned long long *)dev_alloc(c, (size_t)m * 8);
  int64_t *v2 = (int64_t *)dev_alloc(c, (size_t)m * 8);
  int64_t *vs = (int64_t *)dev_alloc(c, (size_t)m * 8);
  int64_t *head = (int64_t *)dev_alloc(c, (size_t)m * 8);
  int64_t *pos = (int64_t *)dev_alloc(c, (size_t)m * 8);
  void *tmp = dev_alloc(c, tb);
  unsigned long long *ukeys = nullptr;
  int rc = CC_OK;
  do {
    if (!k2 || !ks || !v2 || !vs || !head || !pos || !tmp) { rc = CC_ERR_OOM; break; }
    if ((int64_t)(int)m != m) { rc = CC_ERR_OOM; break; }  // one sort covers the list
    k_pair_expand<<<grid_for(n_pairs), 256, 0, st>>>(keys, n_pairs, k2, v2);
    c.kernels++;
    size_t t1 = tb;
    if (cub::DeviceRadixSort::SortPairs(tmp, t1, k2, ks, v2, vs, (int)m, 0, 64, st) != cudaSuccess) {
      rc = CC_ERR_CUDA;
      break;
    }
    k_pair_heads<<<grid_for(m), 256, 0, st>>>(ks, m, head);
    c.kernels++;
    size_t t2 = tb;
    if (cub::DeviceScan::ExclusiveSum(tmp, t2, head, pos, (int)m, st) != cudaSuccess) { rc = CC_ERR_CUDA; break; }
    int64_t last[2] = {0, 0};
    if (cudaMemcpyAsync(&last[0], pos + m - 1, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&last[1], head + m - 1, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rc = CC_ERR_CUDA;
      break;
    }
    pg.nnz = last[0] + last[1];
    pg.col = (int32_t *)dev_alloc(c, (size_t)pg.nnz * 4);
    pg.rev = (int64_t *)dev_alloc(c, (size_t)pg.nnz * 8);
    pg.ridx = (int64_t *)dev_alloc(c, (size_t)pg.nnz * 8);
    ukeys = (unsigned long long *)dev_alloc(c, (size_t)pg.nnz * 8);
    if (!pg.col || !pg.rev || !pg.ridx || !ukeys) { rc = CC_ERR_OOM; break; }
    k_pair_scatter<<<grid_for(m), 256, 0, st>>>(ks, vs, pos, m, pg.col, ukeys, pg.ridx);
    k_pair_rows<<<grid_for(n + 1), 256, 0, st>>>(ukeys, pg.nnz, n, pg.row);
    k_pair_lo<<<grid_for(n), 256, 0, st>>>(pg.row, pg.col, n, pg.lo_cnt);
    k_pair_rev<<<grid_for(pg.nnz), 256, 0, st>>>(ukeys, pg.row, pg.col, pg.nnz, pg.rev);
    c.kernels += 4;
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) rc = CC_ERR_CUDA;
  } while (false);
  cudaStreamSynchronize(st);
  dev_free(c, k2, (size_t)m * 8);
  dev_free(c, ks, (size_t)m * 8);
  dev_free(c, v2, (size_t)m * 8);
  dev_free(c, vs, (size_t)m * 8);
  dev_free(c, head, (size_t)m * 8);
  dev_free(c, pos, (size_t)m * 8);
  dev_free(c, tmp, tb);
  dev_free(c, ukeys, (size_t)std::max<int64_t>(pg.nnz, 1) * 8);
  return rc;
}

int pair_rows_by_position(Ctx &c, const PairGraph &pg, u64 *dense) {
  if (pg.nnz == 0) return CC_OK;
  k_pair_dense<<<grid_for(pg.nnz * pg.R), 256, 0, c.stream>>>(pg.ridx, pg.rows, pg.nnz, pg.R, dense);
  c.kernels++;
  return cudaGetLastError() == cudaSuccess ? CC_OK : CC_ERR_CUDA;
}

}  // namespace cc
