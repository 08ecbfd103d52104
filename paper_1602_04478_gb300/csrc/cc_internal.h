// Internal declarations shared by the library's host translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "../../include/cc.h"

namespace cc {

constexpr int kMaxK = CC_MAX_K;
constexpr int kMaxCycle = 8;  // longest root cycle the closure kernel handles
constexpr int kMaxPairGraphs = 4;  // pair-keyed edge tables one cycle block may read
// levels (hops) of the longer half the cycle kernel walks; a Case-2 block
// cut at its boundary nodes has halves of d and L - d hops
constexpr int kMaxHalf = kMaxCycle / 2 + 1;

// ------------------------------- query plan -------------------------------
enum StageKind { ST_LEAF = 0, ST_TRI = 1, ST_CYCLE_ROOT = 2, ST_ROOT_NODE = 3, ST_CYCLE_NONROOT = 4 };

// One block of the decomposition tree (Section 4.1) in contraction order.
struct Stage {
  int kind = 0;
  int L = 0;                 // leaf: 2 (a, b); triangle: 3; root cycle: L
  int nodes[kMaxK];          // leaf: a (boundary), b (leaf); cycle in cyclic order
  int nb = 0;                // boundary nodes of the block (0, 1 or 2)
  int bd[2] = {-1, -1};      // ordered: a 2-boundary table is keyed (img bd0 -> img bd1)
  int node_child[kMaxK];     // per position: stage index of the annotating block, -1 none
  int edge_child[kMaxK];     // per cycle edge nodes[i] -> nodes[i+1 mod L]
  bool edge_fwd[kMaxK];      // child's first boundary node is nodes[i]
  // Case-2 table keyed by pairs that need not be data edges (the boundary
  // nodes are not adjacent in the cycle, or joined by such an edge)
  bool pair_out = false;
  int s = 0;                 // |SQ(B)|: query nodes of the represented subquery
  uint32_t sq_mask = 0;
  std::string sig;           // structure of the block's subtree: equal strings, equal tables
};

struct Plan {
  int k = 0;
  std::vector<std::pair<int, int>> edges;
  std::vector<Stage> stages;  // children before parents; the last stage is the root
  int64_t aut = 0;
  int longest_cycle = 0;
  bool supported = false;
};

// Builds the default plan (searching decomposition orders) or applies an
// explicit order.  Returns a CC_ status code.
// paper_only: rank trees by the paper's factors alone (Section 5.3), without
// the library's engine-aware cost factor
int plan_query(int k, const std::vector<std::pair<int, int>> &edges, Plan &out, bool paper_only = false);
int plan_explicit(int k, const std::vector<std::pair<int, int>> &edges,
                  const std::vector<int> &block_seq, Plan &out);
int64_t count_automorphisms(int k, const std::vector<std::pair<int, int>> &edges);

// One decomposition tree: its contraction sequence (cc_set_decomposition's
// block_seq) and the paper's ranking factors (Section 5.3).
struct PlanChoice {
  std::vector<int> seq;
  bool supported = false, is_default = false, is_paper = false;
  int longest = 0, boundary = 0, annotations = 0;
  double cost = 0;  // the library's engine-aware join cost
};
int plan_enumerate(int k, const std::vector<std::pair<int, int>> &edges, std::vector<PlanChoice> &out);
// Edge i of stage g is annotated by a pair-keyed table (walked over its pair graph).
inline bool edge_pair_keyed(const std::vector<Stage> &st, const Stage &g, int i) {
  return g.edge_child[i] >= 0 && st[g.edge_child[i]].pair_out;
}

// Structural work of one stage of a colouring pass (independent of the
// colouring): edge-subset updates, algorithmic bytes (the compulsory reads
// and writes of its kernels) and, for a root cycle, the data edges scanned
// out of each level (both halves).
struct StageWork {
  int kind = 0;
  double units = 0, bytes = 0;
  double scans[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};

// ------------------------------- data graph -------------------------------
struct DevGraph {
  bool owned = true;          // false: device arrays belong to another context (shared graph)
  int64_t n = 0, nnz = 0, max_deg = 0;
  int64_t *row = nullptr;     // [n+1]  relabelled CSR (vertex = degree rank)
  int32_t *col = nullptr;     // [nnz]  neighbour ranks, each row ascending
  int64_t *rev = nullptr;     // [nnz]  position of the reverse directed edge
  int32_t *lo_cnt = nullptr;  // [n]    neighbours with a smaller rank (a row prefix)
  int32_t *id_of = nullptr;   // [n]    rank -> caller id
  int32_t *rank_of = nullptr; // [n]    caller id -> rank
  uint8_t *colors = nullptr;  // [T][n] explicit colours in rank order, or null
  int colors_T = 0;
  int colors_max = -1;        // largest explicit colour (must be below the query's k)
  std::vector<int64_t> h_row;  // host copy of the relabelled row pointers
  std::map<int, std::vector<struct StageWork>> work_detail;  // query id -> per-stage structural work
  std::map<int, int> tuned_heavy;    // query id -> heavy-source degree threshold (autotuned)
  std::vector<int64_t> h_push_work;  // per rank u: pairs (v, w), v in N<(u), w in N(v), w < u (empty: not yet)
  // triangle list: every triangle u > v > w once, grouped by u, with the CSR
  // positions of u->v, u->w, v->w (colour-independent, built on first use)
  int tri_state = 0;                 // 0 not built yet, 1 built, -1 above the memory cap
  int64_t n_tri = 0;
  int32_t *tri_u = nullptr, *tri_v = nullptr, *tri_w = nullptr;
  int64_t *tri_p = nullptr;          // [3][n_tri]
  // pair lists of Case-2 blocks: entries of the last pass, by (plan, stage) --
  // the next pass sizes its buffers from it and appends in one launch
  std::map<std::pair<const void *, int>, int64_t> pair_hint;
};

// -------------------------------- context --------------------------------
struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  cc_alloc_fn alloc = nullptr;
  cc_free_fn free_fn = nullptr;
  void *alloc_user = nullptr;
  size_t budget = 0, in_use = 0;
  uint64_t seed = 1;
  std::map<int, DevGraph> graphs;
  std::map<int, Plan> plans;
  int next_graph = 1, next_query = 1;
  // device scratch reused across calls
  uint16_t *lut_rank = nullptr;    // [4096]
  uint16_t *lut_unrank = nullptr;  // [13][924]
  unsigned long long *d_status = nullptr;  // [4]: count lo, overflow flag, timeout flag, spare
  void *scratch = nullptr;
  size_t scratch_bytes = 0;
  uint64_t scratch_layout = 0;   // layout of the cycle kernel's scratch last used
  bool scratch_dirty = true;     // contents unknown (fresh, or a launch failed)
  unsigned epoch = 0;
  void *hv_scratch = nullptr;    // heavy-source cycle scratch (all zero between launches)
  size_t hv_scratch_bytes = 0;
  void *tag_scratch = nullptr;   // colour-tagged adjacency, rewritten every pass (no zero invariant)
  size_t tag_scratch_bytes = 0;
  bool hv_dirty = true;
  const int64_t *cur_graph_row = nullptr;  // host row pointers of the graph being counted
  DevGraph *cur_graph = nullptr;           // the graph being counted
  int heavy_degree = -1;         // sources of at least this degree take the heavy path (-1: tuned / default)
  int procedure = CC_PROC_DB;    // root cycles of length >= 4: DB (degree order) or PS (no order)
  bool tri_list = true;          // triangle blocks stream the graph's triangle list
  int cur_tuned_heavy = -1;      // tuned threshold of the (graph, query) being enqueued, -1 none
  cudaStream_t own_stream = nullptr;  // created for graph capture when the caller's stream is the legacy one
  bool capture = true;           // batches replay a captured CUDA graph
  int batch_lanes = 2;           // concurrent lanes of a batch (this context and batch_lanes - 1 others)
  std::vector<struct cc_ctx *> lanes;  // the other lanes' contexts (own stream and scratch, shared graphs)
  struct BatchCache;
  std::map<std::string, BatchCache *> batches;
  uint64_t kernels = 0;          // kernels launched by this context (a graph replay adds those it holds)
  // timing
  bool timing = false;
  std::map<std::string, std::pair<double, int64_t>> times;
  std::vector<std::pair<std::string, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
};

void *dev_alloc(Ctx &c, size_t bytes);
void dev_free(Ctx &c, void *p, size_t bytes);
int ensure_scratch(Ctx &c, size_t bytes);
int ensure_hv_scratch(Ctx &c, size_t bytes);  // grows and, when fresh or dirty, zeroes the heavy scratch
int ensure_tag_scratch(Ctx &c, size_t bytes); // grows only

// kernel-launch bracketing for the optional timing
void batch_cache_clear(Ctx &c);  // drop captured batch graphs and their buffers
void timing_begin(Ctx &c, const char *name);
void timing_end(Ctx &c);
void timing_flush(Ctx &c);

}  // namespace cc

// the opaque handle of the C-ABI
struct cc_ctx {
  cc::Ctx c;
};
