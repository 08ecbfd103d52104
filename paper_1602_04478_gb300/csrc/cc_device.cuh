// Device helpers shared by the library's kernels.
//
// Signatures (Section 4.2, "Signature") are colour sets, stored as masks
// (bit c = colour c, k <= 12).  Projection-table rows are dense over the
// signatures a row can hold:
//   * unary row of vertex x (signature size s, always containing chi(x)):
//     slot = colex rank of the mask with chi(x)'s bit squeezed out, among
//     (s-1)-subsets of the other k-1 colours -> C(k-1, s-1) slots;
//   * pair row of (x, y) (containing chi(x) and chi(y), chi(x) != chi(y)):
//     both bits squeezed out -> C(k-2, s-2) slots.
// The colex rank of a mask with bits p_0 < p_1 < ... is sum_i C(p_i, i+1);
// ranks of j-subsets are 0 .. C(m, j)-1 inside any universe of m >= max
// bit + 1 colours.  rank/unrank come from lookup tables built at start-up.
#pragma once
#include <cstdint>

namespace cc {

constexpr int kUnrankStride = 924;  // C(12, 6): most masks of one popcount

struct Lut {
  const uint16_t *rank;    // [4096]   colex rank within the popcount class
  const uint16_t *unrank;  // [13][924] mask of (popcount, rank)
};

__device__ __forceinline__ uint32_t squeeze1(uint32_t m, int c) {
  return (m & ((1u << c) - 1u)) | ((m >> (c + 1)) << c);
}
__device__ __forceinline__ uint32_t expand1(uint32_t m, int c) {
  return (m & ((1u << c) - 1u)) | ((m >> c) << (c + 1)) | (1u << c);
}
__device__ __forceinline__ uint32_t squeeze2(uint32_t m, int a, int b) {
  int hi = a > b ? a : b, lo = a > b ? b : a;
  return squeeze1(squeeze1(m, hi), lo);
}
__device__ __forceinline__ uint32_t expand2(uint32_t m, int a, int b) {
  int hi = a > b ? a : b, lo = a > b ? b : a;
  return expand1(expand1(m, lo), hi);
}
__device__ __forceinline__ int lut_rank(const Lut &L, uint32_t m) { return __ldg(L.rank + m); }
__device__ __forceinline__ uint32_t lut_unrank(const Lut &L, int pop, int r) {
  return __ldg(L.unrank + pop * kUnrankStride + r);
}
// slot of mask m in a unary row of a vertex coloured c
__device__ __forceinline__ int uslot(const Lut &L, uint32_t m, int c) { return lut_rank(L, squeeze1(m, c)); }
// mask of slot r in a unary row of size-s signatures of a vertex coloured c
__device__ __forceinline__ uint32_t umask(const Lut &L, int s, int r, int c) {
  return expand1(lut_unrank(L, s - 1, r), c);
}
__device__ __forceinline__ int pslot(const Lut &L, uint32_t m, int a, int b) {
  return lut_rank(L, squeeze2(m, a, b));
}
__device__ __forceinline__ uint32_t pmask(const Lut &L, int s, int r, int a, int b) {
  return expand2(lut_unrank(L, s - 2, r), a, b);
}

// ---------------- exact uint64 arithmetic with overflow detection ----------------
__device__ __forceinline__ unsigned long long mul_ck(unsigned long long a, unsigned long long b,
                                                     unsigned &ovf) {
  ovf |= (__umul64hi(a, b) != 0ull);
  return a * b;
}
__device__ __forceinline__ unsigned long long add_ck(unsigned long long a, unsigned long long b,
                                                     unsigned &ovf) {
  unsigned long long r = a + b;
  ovf |= (r < a);
  return r;
}
__device__ __forceinline__ void atomic_add_ck(unsigned long long *p, unsigned long long v, unsigned &ovf) {
  if (v == 0ull) return;
  unsigned long long old = atomicAdd(p, v);
  ovf |= (old + v < old);
}
// warp sum of uint64 values with overflow detection (all lanes get the sum)
__device__ __forceinline__ unsigned long long warp_sum_ck(unsigned long long v, unsigned &ovf) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = add_ck(v, w, ovf);
  }
  return v;
}

// status words in device memory
// ST_SCAN0 + j: data edges scanned out of level j of a root cycle's halves
// (structural counting only; a status block then has kStatusWords words).
// ST_BOUNDS: an index outside its array (bounds-check build only).
// ST_PAIRCAP: a Case-2 pair list outgrew the buffer sized by its count pass.
enum { ST_COUNT = 0, ST_OVERFLOW = 1, ST_TIMEOUT = 2, ST_BADGRAPH = 3, ST_UNITS = 4, ST_MAXDEG = 5, ST_BOUNDS = 6,
       ST_PAIRCAP = 7, ST_SCAN0 = 8 };
constexpr int kStatusWords = 16;

// Bounds-check build (libcc_boundscheck.so, CC_BOUNDS_CHECK set): an index
// read from data (CSR entries, lists, local indices, triangle records)
// outside its array sets status[ST_BOUNDS] and the access is skipped.  In
// the normal build the check compiles away.
#ifdef CC_BOUNDS_CHECK
__device__ __forceinline__ bool cc_in(int64_t i, int64_t size, unsigned long long *status) {
  if (i >= 0 && i < size) return true;
  atomicOr(status + ST_BOUNDS, 1ull);
  return false;
}
#else
__device__ __forceinline__ bool cc_in(int64_t, int64_t, unsigned long long *) { return true; }
#endif

__device__ __forceinline__ void flag_overflow(unsigned long long *status, unsigned ovf) {
  if (ovf) atomicOr(status + ST_OVERFLOW, 1ull);
}

// True, in every thread of the block, when a count of this pass has already
// exceeded 2^64-1.  The uint64 result is then fixed (UINT64_MAX with
// CC_ERR_OVERFLOW), so the work kernels of the general root-cycle path
// return at once; the kernels that return their scratch to zero still run.
// The flag is read once per block, so the decision is uniform: call it at
// kernel entry, before any divergence, in a 1-D block.
__device__ __forceinline__ bool block_sees_overflow(const unsigned long long *status) {
  __shared__ int s_flag;
  if (threadIdx.x == 0) s_flag = *(const volatile unsigned long long *)(status + ST_OVERFLOW) != 0ull;
  __syncthreads();
  return s_flag != 0;
}

// first index in sorted a[lo, hi) with a[i] >= key
__device__ __forceinline__ int64_t lower_bound_i32(const int32_t *a, int64_t lo, int64_t hi, int32_t key) {
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (__ldg(a + mid) < key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

}  // namespace cc
