// Kernel argument blocks and launchers (host side of each .cu file).
#pragma once
#include "cc_device.cuh"
#include "cc_internal.h"

namespace cc {

typedef unsigned long long u64;

struct GraphView {
  int64_t n = 0, nnz = 0;
  const int64_t *row = nullptr;
  const int32_t *col = nullptr;
  const int64_t *rev = nullptr;
  const int32_t *lo_cnt = nullptr;
};

// unary table [n][R] over signatures of size s (p == nullptr: no annotation)
struct TabU {
  const u64 *p = nullptr;
  int s = 1;
  int R = 1;
};
// edge-keyed table [nnz][R] over size-s signatures; use_rev: the row of a
// traversal x -> y is rev[pos(x -> y)] instead of pos(x -> y).
// gi >= 0 (cycle kernel only): the table is keyed by the positions of the
// pair graph pg[gi] of the cycle's arguments -- a Case-2 block whose boundary
// images need not be adjacent in the data graph -- and the row of position q
// is ridx[q] (-1: an all-zero row)
struct TabE {
  const u64 *p = nullptr;
  int s = 2;
  int R = 1;
  bool use_rev = false;
  int gi = -1;
  const int64_t *ridx = nullptr;
  int64_t nrows = 0;  // rows behind ridx (bounds-check build)
};

struct LeafArgs {
  GraphView g;
  const uint8_t *colors = nullptr;
  int k = 0;
  Lut lut;
  TabU A, B;
  TabE E;
  int sY = 0, RY = 0;  // neighbour aggregate (edge x block at b)
  u64 *out = nullptr;
  int s_out = 0, R_out = 0;
  u64 *status = nullptr;
};

struct TriArgs {
  GraphView g;
  const uint8_t *colors = nullptr;
  int k = 0;
  Lut lut;
  TabU N[3];
  TabE E[3];        // E[i]: triangle edge nodes[i] -> nodes[i+1]; use_rev for that direction
  int nb = 0;       // output: 0 root count, 1 unary at bd0, 2 edge-keyed bd0 -> bd1
  int bd[2] = {-1, -1};  // positions (0..2) of the boundary nodes
  int s_out = 3, R_out = 1;
  u64 *out = nullptr;
  u64 *per_vertex = nullptr;  // root: count by highest vertex (rank order), nullable
  u64 *status = nullptr;
  int *work_counter = nullptr;
  bool count_units = false;   // add the wedges scanned to status[ST_UNITS]
  // the graph's triangle list (n_tri < 0: none; the kernels then scan the wedges)
  int64_t n_tri = -1;
  const int32_t *tri_u = nullptr, *tri_v = nullptr, *tri_w = nullptr;
  const int64_t *tri_p = nullptr;  // [3][n_tri]: CSR positions of u->v, u->w, v->w
};

int launch_leaf(Ctx &c, const LeafArgs &a);
int launch_root_sum(Ctx &c, const GraphView &g, const u64 *table, u64 *per_vertex, u64 *status);
int launch_triangle(Ctx &c, const TriArgs &a);
// Build the graph's triangle list (once; a list above the memory cap is not
// built and the triangle kernels scan wedges instead).  Synchronises.
int tri_list_build(Ctx &c, DevGraph &g);
void tri_list_free(Ctx &c, DevGraph &g);
// Before a plan runs on g: the colouring-independent structure it uses
// (the triangle list when the plan has triangle blocks).  Synchronises;
// never called under stream capture.
int prepare_plan_graph(Ctx &c, DevGraph &g, const Plan &p);

// root cycle (L >= 4) closure; see cycle.cu
struct CycleArgs {
  GraphView g;
  const uint8_t *colors = nullptr;
  int k = 0;
  Lut lut;
  int L = 0;
  TabU N[kMaxCycle];
  TabE Efw[kMaxCycle];   // edge i traversed nodes[i] -> nodes[i+1]
  TabE Ebw[kMaxCycle];   // edge i traversed nodes[i+1] -> nodes[i]
  int multiplier = 1;    // rotations folded into one highest-node choice
  int n_h = 0;
  int hs[kMaxCycle];
  u64 *per_vertex = nullptr;  // count by highest vertex (rank order), nullable
  u64 *status = nullptr;
  bool count_units = false;   // add the structural edge-subset work to status[ST_UNITS]
  int32_t light_end = 0;      // the per-CTA kernel takes sources of rank < light_end
  bool no_order = false;      // PS procedure: paths from u are not restricted to vertices below u
  // length of P+ (the cut nodes are a_h and a_{h+split}); 0: floor(L/2);
  // split_h[h] != 0 overrides it for highest node h
  int split = 0;
  int split_h[kMaxCycle] = {0, 0, 0, 0, 0, 0, 0, 0};
  // pair graphs of the pair-keyed edge tables (TabE::gi)
  GraphView pg[kMaxPairGraphs];
  // Non-root cycle (no_order, the first boundary node at position 0, its
  // image u the source; signatures of size s_out, rows of R_out slots):
  //   out_mode 1: one boundary node; the unary table [n][R_out] by u
  //   out_mode 2: two boundary nodes a_0, a_1 (split 1, the pair is a data
  //               edge); the edge-keyed table [nnz][R_out], row pos(u -> x)
  //   out_mode 3: two boundary nodes a_0, a_split; every nonzero (u, x) row
  //               appended to pair_keys (u << 32 | x) / pair_rows [][R_out]
  //               (pair_keys null: only counted into *pair_count)
  int out_mode = 0;
  // out_mode 1 under DB (Case 1 with the highest node not the boundary):
  // out_key_x[hi], the row of highest-node choice hs[hi] is the meeting
  // vertex x's (the boundary node is the cut node a_{h+split}), added by
  // atomics; out_atomic, u's rows are added rather than stored (other CTAs
  // add to them too)
  bool out_key_x[kMaxCycle] = {false, false, false, false, false, false, false, false};
  bool out_atomic = false;
  u64 *out = nullptr;
  int R_out = 0, s_out = 0;
  unsigned long long *pair_keys = nullptr;
  u64 *pair_rows = nullptr;
  unsigned long long *pair_count = nullptr;
  int64_t pair_cap = 0;
};
// Pair graph of a Case-2 table: the symmetric closure of its (u, x) keys as a
// CSR over the data graph's vertices (rows ascending), with rev and lo_cnt
// like the data graph, and the row index of each position into the rows
// (-1 where only the reverse pair has a row).  Built from the appended list.
struct PairGraph {
  int64_t n = 0, n_pairs = 0, nnz = 0;
  int64_t *row = nullptr;
  int32_t *col = nullptr;
  int64_t *rev = nullptr;
  int32_t *lo_cnt = nullptr;
  int64_t *ridx = nullptr;
  u64 *rows = nullptr;  // [n_pairs][R] in a buffer of rows_cap rows
  int64_t rows_cap = 0;
  int R = 0;
};
int pair_graph_build(Ctx &c, int64_t n, const unsigned long long *keys, int64_t n_pairs, PairGraph &pg);
void pair_graph_free(Ctx &c, PairGraph &pg);
// dense[q][R] = the row of position q (zero where none), for a leaf block's join
int pair_rows_by_position(Ctx &c, const PairGraph &pg, u64 *dense);
int run_heavy(Ctx &c, const CycleArgs &a, int32_t first_rank, int B);
bool plain_cycle_eligible(const CycleArgs &a);
int run_plain_heavy(Ctx &c, const CycleArgs &a, int32_t first_rank);
int run_plain_light(Ctx &c, const CycleArgs &a, int32_t end_rank);

// scratch slots of the per-CTA plain-cycle push kernel (one slot per CTA)
struct PlScratch {
  char *base;
  size_t slot_bytes;
  size_t o_w2, o_w3, o_mark, o_id3, o_l2, o_l3;  // rows by local index; ids by vertex; lists
};
int launch_pc_light_raw(cudaStream_t stream, int L, const GraphView &g, const uint8_t *colors, const PlScratch &S,
                        int slots, int32_t end_rank, int *work, u64 *status, int k);
int heavy_group_size(const CycleArgs &a);
int launch_cycle(Ctx &c, const CycleArgs &a);
size_t cycle_scratch_bytes(const CycleArgs &a, int slots);

// executor (api.cu)
struct Table {
  u64 *p = nullptr;
  size_t bytes = 0;
  int arity = 0;  // 1 unary, 2 edge-keyed
  int s = 0, R = 0;
  bool pair = false;  // pair-keyed (rows in pg.rows, built during the pass)
  PairGraph pg;
};
struct PassBuffers {
  std::vector<Table> T;
  uint8_t *colors = nullptr;
  int *counter = nullptr;
};
int alloc_pass(Ctx &c, const DevGraph &g, const Plan &p, PassBuffers &B);
size_t request_table_bytes(const Plan &p, const DevGraph &g);
void free_pass(Ctx &c, const DevGraph &g, PassBuffers &B);
// detail (nullable): structural counting pass; per-stage work appended (the
// pass synchronises after every stage and needs a status block of
// kStatusWords words)
int enqueue_pass(Ctx &c, DevGraph &g, const Plan &p, int64_t trial, PassBuffers &B, u64 *status, u64 *d_per_vertex,
                 std::vector<StageWork> *detail);
int status_code(const u64 *st);
int run_plan(Ctx &c, DevGraph &g, const Plan &p, int64_t trial, u64 *count, bool *overflow, u64 *d_per_vertex,
             std::vector<StageWork> *detail);

int graph_load(Ctx &c, int64_t n, const int64_t *row_ptr, const int32_t *col, int64_t nnz, DevGraph &g);
void graph_free(Ctx &c, DevGraph &g);
int colors_fill(Ctx &c, const DevGraph &g, int k, int64_t trial, uint8_t *d_out);
int colors_set(Ctx &c, DevGraph &g, const uint8_t *h_colors, int T);
int luts_init(Ctx &c);

inline GraphView view_of(const DevGraph &g) {
  GraphView v;
  v.n = g.n;
  v.nnz = g.nnz;
  v.row = g.row;
  v.col = g.col;
  v.rev = g.rev;
  v.lo_cnt = g.lo_cnt;
  return v;
}

inline int64_t binom(int a, int b) {
  if (b < 0 || a < 0 || b > a) return 0;
  int64_t r = 1;
  for (int i = 1; i <= b; i++) r = r * (a - b + i) / i;
  return r;
}

}  // namespace cc
