// Colourful cycle count that allocates no device memory.
//
// Some callers cannot let a library allocate GPU memory: code running where
// cudaMalloc is unavailable or forbidden (a host that hands out a fixed
// arena, a caller inside its own memory pool, an embedded runtime with no
// allocator).  This entry point serves them.  The caller passes the graph,
// the colours and the output; the kernel's working memory is one file-scope
// __device__ array of kNoAllocScratchBytes (64 MiB), which every GPU that
// loads this library holds until the process exits.
//
// The count is the same one cc_count gives for a plain cycle query C_L,
// L in {4, 5, 6}, k = L: the per-CTA push kernel of the plain-cycle path,
// run with vertex ids as the vertex order (any total order gives the same
// count; the degree order is only faster), so no relabelled copy of the
// graph is needed.
#include <mutex>

#include "cc_kernels.h"

namespace cc {

constexpr size_t kNoAllocScratchBytes = (size_t)64 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

// The host-side name g_noalloc_scratch is only a stand-in for the device
// array; kernels must be given the address cudaGetSymbolAddress returns,
// looked up once per device with that device current.
std::mutex g_mu;
void *g_addr[64] = {nullptr};

int scratch_address(int device, char **out) {
  if (device < 0 || device >= 64) return CC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[device]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return CC_ERR_CUDA;
    }
    g_addr[device] = p;
  }
  *out = (char *)g_addr[device];
  return CC_OK;
}

// lower-neighbour counts (rows must be sorted), input checks, max degree
__global__ void k_na_prepare(int64_t n, const int64_t *row, const int32_t *col, const uint8_t *colors, int k,
                             int32_t *lo_cnt, u64 *status) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = row[v], e = row[v + 1];
    atomicMax(status + ST_MAXDEG, (u64)(e > b ? e - b : 0));
    bool bad = e < b || colors[v] >= k;
    int32_t lo = 0;
    for (int64_t i = b; i < e && !bad; i++) {
      const int32_t c = col[i];
      if (c < 0 || c >= n || c == v || (i > b && col[i - 1] >= c)) bad = true;
      lo += c < v;
    }
    lo_cnt[v] = lo;
    if (bad) atomicOr(status + ST_BADGRAPH, 1ull);
  }
}

}  // namespace
}  // namespace cc

using namespace cc;

extern "C" int cc_count_cycle_noalloc(int device, void *cuda_stream, int L, int64_t n, const int64_t *d_row_ptr,
                                      const int32_t *d_col, const uint8_t *d_colors, uint64_t *count) {
  if (L < 4 || L > 6 || n <= 0 || n >= ((int64_t)1 << 31) || !d_row_ptr || !d_col || !d_colors || !count)
    return CC_ERR_INVALID_ARG;
  // layout inside the static array: status words, work counter, lower
  // counts, then as many per-CTA slots as fit (at least one)
  const size_t head = 256;
  const size_t lo_bytes = ((size_t)n * 4 + 255) & ~(size_t)255;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  PlScratch S;
  S.o_w2 = take((size_t)n * 32);
  S.o_w3 = L >= 5 ? take((size_t)n * 64) : 0;
  S.o_mark = take((size_t)n * 4);
  S.o_id3 = L >= 5 ? take((size_t)n * 4) : 0;
  S.o_l2 = take((size_t)n * 4);
  S.o_l3 = L >= 5 ? take((size_t)n * 4) : 0;
  S.slot_bytes = off;
  if (head + lo_bytes + S.slot_bytes > kNoAllocScratchBytes) return CC_ERR_INVALID_ARG;  // graph too large
  const int slots = (int)std::min<size_t>(64, (kNoAllocScratchBytes - head - lo_bytes) / S.slot_bytes);
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) return CC_ERR_CUDA;
  struct Restore {
    int d;
    ~Restore() { cudaSetDevice(d); }
  } restore{prev};
  char *base = nullptr;
  int rc = scratch_address(device, &base);
  if (rc != CC_OK) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  u64 *status = (u64 *)base;
  int *work = (int *)(base + 128);
  int32_t *lo_cnt = (int32_t *)(base + head);
  S.base = base + head + lo_bytes;
  // everything the kernels accumulate into must start at zero
  const size_t used = head + lo_bytes + (size_t)slots * S.slot_bytes;
  if (cudaMemsetAsync(base, 0, used, st) != cudaSuccess) return CC_ERR_CUDA;
  k_na_prepare<<<152 * 4, 256, 0, st>>>(n, d_row_ptr, d_col, d_colors, L, lo_cnt, status);
  // level-3 entries are u32 sums bounded by deg(x) * deg(u): exact only
  // while the maximum degree is below 2^16
  u64 pre[8];
  if (cudaMemcpyAsync(pre, status, sizeof(pre), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return CC_ERR_CUDA;
  if (pre[ST_BADGRAPH]) return CC_ERR_BAD_GRAPH;
  if (pre[ST_MAXDEG] >= 65536) return CC_ERR_INVALID_ARG;
  GraphView g;
  g.n = n;
  g.row = d_row_ptr;
  g.col = d_col;
  g.lo_cnt = lo_cnt;
  rc = launch_pc_light_raw(st, L, g, d_colors, S, slots, (int32_t)n, work, status, L);
  if (rc != CC_OK) return rc;
  u64 h[4] = {0, 0, 0, 0};
  if (cudaMemcpyAsync(h, status, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return CC_ERR_CUDA;
  if (h[ST_BADGRAPH]) return CC_ERR_BAD_GRAPH;
  // a bounded wait that gave up skipped a contribution: the count is incomplete
  if (h[ST_TIMEOUT]) return CC_ERR_TIMEOUT;
  if (h[ST_OVERFLOW]) {
    *count = UINT64_MAX;
    return CC_ERR_OVERFLOW;
  }
  *count = h[ST_COUNT];
  return CC_OK;
}
