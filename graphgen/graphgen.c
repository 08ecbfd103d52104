/*
 * Seeded synthetic data-graph generators (test and benchmark inputs only).
 *
 * This module holds no part of the colour-coding method: it only draws simple
 * undirected graphs and writes them as a symmetric CSR (int64 row pointers,
 * int32 column ids, every row sorted ascending, no self-loops, no duplicate
 * edges).  Both the CPU oracle and the CUDA library consume its output.
 *
 * Random numbers come from SplitMix64 (Steele, Lea, Flood 2014; the output
 * function is Vigna's published mix), used as a counter-based generator:
 * draw i of stream s is mix(key(seed, s) + (i + 1) * golden).
 *
 * Families:
 *   - Erdos-Renyi G(n, m): m distinct non-loop pairs by rejection.
 *   - Chung-Lu: edge (u, v) independently with probability w_u w_v / sum(w)
 *     (the random power-law model the paper analyses in its Section 7), with
 *     w_i proportional to (i + 1)^(-1/(gamma - 1)), rescaled to a target mean
 *     degree and capped at sqrt(sum w) so every probability is at most 1.
 *     Exact O(n + m) sampling by the skipping method of Miller and Hagberg
 *     ("Efficient generation of networks with given expected degrees", 2011).
 *   - R-MAT (Chakrabarti, Zhan, Faloutsos 2004): 2^scale vertices,
 *     edge_factor * 2^scale recursive quadrant draws with 16-bit integer
 *     thresholds, then symmetrised and deduplicated.
 * Chung-Lu and R-MAT apply a seeded random relabelling of vertex ids at the
 * end, so ids carry no degree information.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Counter-based draw: the i-th SplitMix64 output of a stream whose state
 * starts at mix64(seed) ^ stream. */
static inline uint64_t draw(uint64_t seed, uint64_t stream, uint64_t i) {
  uint64_t state = mix64(seed + GOLDEN) ^ (stream * 0xD1B54A32D192ED03ULL);
  return mix64(state + (i + 1) * GOLDEN);
}

static inline double unit(uint64_t r) { /* in (0, 1] */
  return ((double)(r >> 11) + 1.0) * (1.0 / 9007199254740992.0);
}

/* ---------- LSD radix sort of uint64 keys (stable, 16-bit digits) ---------- */
static int radix_sort_u64(uint64_t *a, int64_t len, int key_bits) {
  if (len <= 1) return 0;
  uint64_t *tmp = (uint64_t *)malloc((size_t)len * sizeof(uint64_t));
  if (!tmp) return -1;
  int64_t *cnt = (int64_t *)malloc(65537 * sizeof(int64_t));
  if (!cnt) { free(tmp); return -1; }
  uint64_t *src = a, *dst = tmp;
  for (int shift = 0; shift < key_bits; shift += 16) {
    memset(cnt, 0, 65537 * sizeof(int64_t));
    for (int64_t i = 0; i < len; i++) cnt[((src[i] >> shift) & 0xFFFF) + 1]++;
    for (int d = 0; d < 65536; d++) cnt[d + 1] += cnt[d];
    for (int64_t i = 0; i < len; i++) dst[cnt[(src[i] >> shift) & 0xFFFF]++] = src[i];
    uint64_t *t = src; src = dst; dst = t;
  }
  if (src != a) memcpy(a, src, (size_t)len * sizeof(uint64_t));
  free(tmp);
  free(cnt);
  return 0;
}

static int bits_for(int64_t n) {
  int b = 1;
  while (((int64_t)1 << b) < n) b++;
  return b;
}

/* Turn a list of undirected pairs (any order, loops/duplicates allowed) into
 * a symmetric deduplicated CSR.  Pairs are packed as (a << 32 | b).
 * On success *row_ptr (n+1) and *col (nnz) are malloc'd. */
static int pairs_to_csr(int64_t n, uint64_t *pairs, int64_t np, int64_t **row_ptr_out,
                        int32_t **col_out, int64_t *nnz_out) {
  /* directed copies, packed with the vertex-id bit width so the sort is short */
  int vb = bits_for(n);
  uint64_t *dir = (uint64_t *)malloc((size_t)(2 * np + 1) * sizeof(uint64_t));
  if (!dir) return -1;
  int64_t nd = 0;
  for (int64_t i = 0; i < np; i++) {
    uint64_t a = pairs[i] >> 32, b = pairs[i] & 0xFFFFFFFFULL;
    if (a == b) continue;
    dir[nd++] = (a << vb) | b;
    dir[nd++] = (b << vb) | a;
  }
  if (radix_sort_u64(dir, nd, 2 * vb) != 0) { free(dir); return -1; }
  int64_t *rp = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
  if (!rp) { free(dir); return -1; }
  int64_t w = 0;
  for (int64_t i = 0; i < nd; i++) {
    if (i > 0 && dir[i] == dir[i - 1]) continue;
    dir[w++] = dir[i];
  }
  int32_t *col = (int32_t *)malloc((size_t)(w > 0 ? w : 1) * sizeof(int32_t));
  if (!col) { free(dir); free(rp); return -1; }
  uint64_t mask = (vb >= 64) ? ~0ULL : ((1ULL << vb) - 1);
  for (int64_t i = 0; i < w; i++) {
    int64_t a = (int64_t)(dir[i] >> vb);
    col[i] = (int32_t)(dir[i] & mask);
    rp[a + 1]++;
  }
  for (int64_t v = 0; v < n; v++) rp[v + 1] += rp[v];
  free(dir);
  *row_ptr_out = rp;
  *col_out = col;
  *nnz_out = w;
  return 0;
}

/* Seeded Fisher-Yates permutation of 0..n-1. */
static int32_t *random_perm(int64_t n, uint64_t seed, uint64_t stream) {
  int32_t *p = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  if (!p) return NULL;
  for (int64_t i = 0; i < n; i++) p[i] = (int32_t)i;
  for (int64_t i = n - 1; i > 0; i--) {
    uint64_t r = draw(seed, stream, (uint64_t)i);
    int64_t j = (int64_t)(((unsigned __int128)r * (unsigned __int128)(i + 1)) >> 64);
    int32_t t = p[i]; p[i] = p[j]; p[j] = t;
  }
  return p;
}

static void relabel_pairs(uint64_t *pairs, int64_t np, const int32_t *perm) {
  for (int64_t i = 0; i < np; i++) {
    uint64_t a = pairs[i] >> 32, b = pairs[i] & 0xFFFFFFFFULL;
    pairs[i] = ((uint64_t)(uint32_t)perm[a] << 32) | (uint64_t)(uint32_t)perm[b];
  }
}

/* ------------------------------ Erdos-Renyi ------------------------------ */
int gg_erdos_renyi(int64_t n, int64_t m, uint64_t seed, int64_t **row_ptr, int32_t **col,
                   int64_t *nnz) {
  if (n < 2 || m < 0 || m > n * (n - 1) / 2) return -2;
  /* open-addressing set of accepted pairs */
  int64_t cap = 1;
  while (cap < 2 * m + 16) cap <<= 1;
  uint64_t *set = (uint64_t *)malloc((size_t)cap * sizeof(uint64_t));
  uint64_t *pairs = (uint64_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(uint64_t));
  if (!set || !pairs) { free(set); free(pairs); return -1; }
  memset(set, 0xFF, (size_t)cap * sizeof(uint64_t));
  int64_t got = 0;
  uint64_t i = 0;
  while (got < m) {
    uint64_t ra = draw(seed, 1, i++), rb = draw(seed, 1, i++);
    uint64_t a = (uint64_t)(((unsigned __int128)ra * (unsigned __int128)n) >> 64);
    uint64_t b = (uint64_t)(((unsigned __int128)rb * (unsigned __int128)n) >> 64);
    if (a == b) continue;
    if (a > b) { uint64_t t = a; a = b; b = t; }
    uint64_t key = (a << 32) | b;
    uint64_t h = mix64(key) & (uint64_t)(cap - 1);
    int dup = 0;
    while (set[h] != ~0ULL) {
      if (set[h] == key) { dup = 1; break; }
      h = (h + 1) & (uint64_t)(cap - 1);
    }
    if (dup) continue;
    set[h] = key;
    pairs[got++] = key;
  }
  free(set);
  int rc = pairs_to_csr(n, pairs, m, row_ptr, col, nnz);
  free(pairs);
  return rc;
}

/* ------------------------------- Chung-Lu ------------------------------- */
/* Expected-degree weights, sorted descending (index 0 is the heaviest). */
static void chung_lu_weights(int64_t n, double mean_deg, double gamma, double *w) {
  double expo = 1.0 / (gamma - 1.0);
  for (int64_t i = 0; i < n; i++) w[i] = pow((double)(i + 1), -expo);
  /* rescale to the target mean, cap at sqrt(sum), repeat until stable */
  for (int it = 0; it < 60; it++) {
    double s = 0.0;
    for (int64_t i = 0; i < n; i++) s += w[i];
    double scale = mean_deg * (double)n / s;
    for (int64_t i = 0; i < n; i++) w[i] *= scale;
    double cap = sqrt(mean_deg * (double)n);
    for (int64_t i = 0; i < n; i++)
      if (w[i] > cap) w[i] = cap;
  }
}

int gg_chung_lu(int64_t n, double mean_deg, double gamma, uint64_t seed, int64_t **row_ptr,
                int32_t **col, int64_t *nnz) {
  if (n < 2 || mean_deg <= 0.0 || gamma <= 1.0) return -2;
  double *w = (double *)malloc((size_t)n * sizeof(double));
  if (!w) return -1;
  chung_lu_weights(n, mean_deg, gamma, w);
  double s = 0.0;
  for (int64_t i = 0; i < n; i++) s += w[i];
  int64_t cap = (int64_t)(0.5 * s * 1.2) + 1024, np = 0;
  uint64_t *pairs = (uint64_t *)malloc((size_t)cap * sizeof(uint64_t));
  if (!pairs) { free(w); return -1; }
  /* Miller-Hagberg: for each u, walk v = u+1.. with geometric skips at the
   * current (non-increasing) probability p, then accept with q/p. */
  for (int64_t u = 0; u + 1 < n; u++) {
    int64_t v = u + 1;
    double p = w[u] * w[v] / s;
    if (p > 1.0) p = 1.0;
    uint64_t ctr = 0;
    while (v < n && p > 0.0) {
      if (p != 1.0) {
        double r = unit(draw(seed, 2 + (uint64_t)u, ctr++));
        v += (int64_t)floor(log(r) / log1p(-p));
      }
      if (v < n) {
        double q = w[u] * w[v] / s;
        if (q > 1.0) q = 1.0;
        double r = unit(draw(seed, 2 + (uint64_t)u, ctr++));
        if (r <= q / p) {
          if (np == cap) {
            cap = cap * 3 / 2 + 1024;
            uint64_t *np2 = (uint64_t *)realloc(pairs, (size_t)cap * sizeof(uint64_t));
            if (!np2) { free(pairs); free(w); return -1; }
            pairs = np2;
          }
          pairs[np++] = ((uint64_t)u << 32) | (uint64_t)v;
        }
        p = q;
        v += 1;
      }
    }
  }
  free(w);
  int32_t *perm = random_perm(n, seed, 1);
  if (!perm) { free(pairs); return -1; }
  relabel_pairs(pairs, np, perm);
  free(perm);
  int rc = pairs_to_csr(n, pairs, np, row_ptr, col, nnz);
  free(pairs);
  return rc;
}

/* --------------------------------- R-MAT --------------------------------- */
int gg_rmat(int scale, int64_t edge_factor, double a, double b, double c, uint64_t seed,
            int64_t **row_ptr, int32_t **col, int64_t *nnz) {
  if (scale < 1 || scale > 30 || edge_factor < 1) return -2;
  int64_t n = (int64_t)1 << scale, m = edge_factor * n;
  uint32_t ta = (uint32_t)(a * 65536.0 + 0.5);
  uint32_t tb = ta + (uint32_t)(b * 65536.0 + 0.5);
  uint32_t tc = tb + (uint32_t)(c * 65536.0 + 0.5);
  uint64_t *pairs = (uint64_t *)malloc((size_t)m * sizeof(uint64_t));
  if (!pairs) return -1;
  for (int64_t e = 0; e < m; e++) {
    uint64_t r = 0, row = 0, colv = 0;
    int avail = 0;
    uint64_t ctr = 0;
    for (int lvl = 0; lvl < scale; lvl++) {
      if (avail == 0) { r = draw(seed, 3 + (uint64_t)e, ctr++); avail = 4; }
      uint32_t x = (uint32_t)(r & 0xFFFF);
      r >>= 16;
      avail--;
      uint64_t bi = 0, bj = 0;
      if (x < ta) { bi = 0; bj = 0; }
      else if (x < tb) { bi = 0; bj = 1; }
      else if (x < tc) { bi = 1; bj = 0; }
      else { bi = 1; bj = 1; }
      row = (row << 1) | bi;
      colv = (colv << 1) | bj;
    }
    pairs[e] = (row << 32) | colv;
  }
  int32_t *perm = random_perm(n, seed, 1);
  if (!perm) { free(pairs); return -1; }
  relabel_pairs(pairs, m, perm);
  free(perm);
  int rc = pairs_to_csr(n, pairs, m, row_ptr, col, nnz);
  free(pairs);
  return rc;
}

/* -------------------- explicit edge list (tests, fixtures) -------------------- */
int gg_from_edges(int64_t n, const int32_t *edges, int64_t n_edges, int64_t **row_ptr,
                  int32_t **col, int64_t *nnz) {
  uint64_t *pairs = (uint64_t *)malloc((size_t)(n_edges > 0 ? n_edges : 1) * sizeof(uint64_t));
  if (!pairs) return -1;
  for (int64_t i = 0; i < n_edges; i++) {
    int32_t a = edges[2 * i], b = edges[2 * i + 1];
    if (a < 0 || b < 0 || a >= n || b >= n) { free(pairs); return -2; }
    pairs[i] = ((uint64_t)(uint32_t)a << 32) | (uint64_t)(uint32_t)b;
  }
  int rc = pairs_to_csr(n, pairs, n_edges, row_ptr, col, nnz);
  free(pairs);
  return rc;
}

void gg_free(void *p) { free(p); }
