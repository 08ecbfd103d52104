/*
 * cc.h -- C-ABI of the GB300 colour-coding library for counting colourful
 * matches of treewidth-2 query graphs (Chakaravarthy, Kapralov, Murali,
 * Petrini, Que, Sabharwal, Schieber: "Subgraph Counting: Color Coding Beyond
 * Trees", arXiv 1602.04478).
 *
 * The library keeps data graphs and per-query plans resident on one CUDA
 * device and runs every step of the count in its own sm_103a kernels.  All
 * pointers in this header are HOST pointers unless a name says "device".
 * Every call is synchronous with respect to the host: results are in the
 * caller's buffers when the call returns.  Calls on one context must not
 * overlap (one host thread at a time per context).
 *
 * Problem (Section 2): for a query Q on k nodes and a data graph G, a match is
 * an injective map pi: V_Q -> V_G with every query edge on a data edge.
 * Given a colouring chi: V_G -> {0..k-1}, a match is colourful when its k
 * images carry k distinct colours.  n_colorful(G, Q, chi) is the number of
 * colourful matches; (k^k / k!) * E_chi[n_colorful] equals the number of
 * matches, and dividing by aut(Q) counts subgraphs (Section 2, "Approximate
 * subgraph counting via color coding").
 *
 * Colouring (the paper leaves the generator open): colour of vertex v
 * (caller's id) in trial t under seed s is
 *     hi64( mix(s ^ (G * (t + 1)) ^ mix(v)) * k ),
 * where G = 0x9E3779B97F4A7C15, mix(x) is SplitMix64's output for state x
 * (z = x + G; z = (z ^ z>>30) * 0xBF58476D1CE4E5B9;
 *  z = (z ^ z>>27) * 0x94D049BB133111EB; z ^ z>>31) and hi64 the upper 64
 * bits of the 128-bit product.  cc_set_colors replaces it with explicit
 * colours.
 *
 * Error behaviour: every int-returning call returns CC_OK (0) or one of the
 * negative CC_ERR_* codes below and leaves outputs it could not compute
 * untouched unless stated.  cc_strerror gives a one-line message.
 */
#ifndef CC_H
#define CC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CC_OK 0
#define CC_ERR_INVALID_ARG (-1)  /* null pointer, out-of-range id or size     */
#define CC_ERR_BAD_GRAPH (-2)    /* CSR not symmetric, self-loop, duplicate    */
#define CC_ERR_NOT_TW2 (-3)      /* query has no block decomposition (tw > 2)  */
#define CC_ERR_K_RANGE (-4)      /* k outside [2, 12]                          */
#define CC_ERR_OOM (-5)          /* device memory would exceed the budget      */
#define CC_ERR_OVERFLOW (-6)     /* a count exceeded 2^64-1 (never wrapped)    */
#define CC_ERR_TIMEOUT (-7)      /* a bounded device wait gave up              */
#define CC_ERR_CUDA (-8)         /* a CUDA runtime call failed                 */
#define CC_ERR_UNSUPPORTED (-9)  /* the query needs a block kind not built    */
#define CC_ERR_NOT_CONNECTED (-10) /* the query graph is not connected         */
#define CC_ERR_BOUNDS (-11)      /* an index left its array (bounds-check build only) */

#define CC_MAX_K 12

typedef struct cc_ctx cc_ctx;

/* Device-memory allocator hooks.  alloc returns a device pointer of at least
 * `bytes` bytes (16-byte aligned) or NULL; free releases it.  Without hooks
 * the library uses cudaMalloc / cudaFree. */
typedef void *(*cc_alloc_fn)(size_t bytes, void *user);
typedef void (*cc_free_fn)(void *ptr, size_t bytes, void *user);

/* Create a context on CUDA device `device` that issues all work on
 * `cuda_stream` (a cudaStream_t; NULL means the legacy default stream).
 * The context owns every device buffer it allocates. */
int cc_create(cc_ctx **out, int device, void *cuda_stream);
void cc_destroy(cc_ctx *ctx);
int cc_set_allocator(cc_ctx *ctx, cc_alloc_fn alloc, cc_free_fn free_fn, void *user);
/* Upper bound on the device bytes the context may hold (0 = no limit).
 * A count whose tables would exceed it fails with CC_ERR_OOM before any
 * launch. */
int cc_set_memory_budget(cc_ctx *ctx, size_t bytes);

/* Heavy/light split of the root-cycle closure: sources (highest cycle
 * vertices) of degree >= `degree` are processed in groups by the whole GPU,
 * the others one per CTA.  -1 restores the library's choice.  The split
 * changes only the speed, never the counts. */
int cc_set_heavy_degree(cc_ctx *ctx, int degree);

/* Procedure for root cycle blocks of length >= 4 and for non-root cycle
 * blocks of length 4-6 with one boundary node (Section 5).
 * CC_PROC_DB (default): the degree-based procedure -- matches split by the
 * cycle node holding the highest vertex in the degree order (Eq. 1), paths
 * extended only through lower vertices (Procedures 1-2, general-cycle
 * figure).  CC_PROC_PS: the path-splitting procedure without vertex order
 * -- one split of the cycle at a_0 and its opposite node, paths extended
 * through any vertex (Procedures 1-2 of the PS algorithm figure).  Both give
 * the same counts; PS does far more work on skewed graphs and runs on the
 * library's general per-source kernel only.  cc_count_per_vertex splits a
 * PS count by the image of a_0.  A non-root cycle with one boundary node b
 * under DB: each node as the highest, cut there and at b; under PS (and for
 * cycles of 7 or 8 nodes): one split at b and its opposite node, no order.
 * Triangle and leaf blocks, and non-root cycles with two boundary nodes
 * (cut at both, no order), are the same under both. */
/* Triangle blocks (enable = 1, the default): the graph's triangles are
 * listed once, on the first count of a query with a triangle block (every
 * triangle u > v > w in the degree order, with the positions of its edges;
 * colour-independent), and every colouring streams that list.  The list is
 * not built when it would take more than a quarter of the memory left to
 * the context; the triangle kernels then scan the wedges of every source
 * each colouring, as they do with enable = 0.  Counts are the same. */
int cc_set_triangle_list(cc_ctx *ctx, int enable);

#define CC_PROC_DB 0
#define CC_PROC_PS 1
int cc_set_procedure(cc_ctx *ctx, int procedure);

/* Copy a data graph to the device.  row_ptr[n+1] (int64) and col[nnz]
 * (int32, caller's vertex ids) describe a symmetric simple graph: each
 * undirected edge appears in both rows, no self-loops, no duplicates.
 * Anything else fails with CC_ERR_BAD_GRAPH (no silent repair).  The caller
 * keeps ownership of its arrays.  The library orders vertices by
 * (degree, id) ascending -- the degree order of Section 5.1 -- and stores the
 * graph relabelled by that rank. */
int cc_load_csr(cc_ctx *ctx, int64_t n, const int64_t *row_ptr, const int32_t *col,
                int64_t nnz, int32_t *graph_id);
int cc_free_graph(cc_ctx *ctx, int32_t graph_id);
int cc_graph_info(cc_ctx *ctx, int32_t graph_id, int64_t *n, int64_t *nnz, int64_t *max_degree);

/* Register a query: k nodes (2..12) and n_edges edges as pairs
 * edges[2i], edges[2i+1] in 0..k-1.  The query must be simple and
 * connected.  The library decomposes it into blocks (Section 4.1: leaf
 * edges and induced cycles with at most two boundary nodes, contracted by
 * Cases 1-3) and computes aut(Q) by enumeration.  CC_ERR_NOT_TW2 when no
 * decomposition exists (Lemma 4.1), CC_ERR_UNSUPPORTED when no
 * decomposition can run (cc_plan_supported: a cycle longer than 8, a Case-2
 * cycle whose longer side between its boundary nodes has more than 5 edges).
 * Non-root cycles of length >= 4 are built from the general per-source
 * kernel: with one boundary node (Case 1) by the procedure cc_set_procedure
 * selects; with two (Case 2) cut at both without vertex order, their table
 * keyed by data edges when the boundary pair is joined by one, else by the
 * nonzero pairs (a pair graph the parent block walks). */
int cc_set_query(cc_ctx *ctx, int k, int n_edges, const int32_t *edges, int32_t *query_id);

/* Replace the query's decomposition by an explicit contraction order.
 * block_seq is a list of records, one per contracted block, in order:
 *   0, a, b          leaf edge (a, b) whose node b has degree one
 *   L, a0, .., aL-1  induced cycle of length L >= 3 in cyclic order
 * The final block (root cycle or single node) is implied.  Each record
 * must name a block of the partly contracted query at that point, else
 * CC_ERR_INVALID_ARG.  Every valid order gives the same counts (Section 5.2);
 * the order only changes the work. */
int cc_set_decomposition(cc_ctx *ctx, int32_t query_id, const int32_t *block_seq, int len);

/* Host-only (no context, no device): the decomposition the library would
 * use for a query, with an optional explicit order (block_seq as for
 * cc_set_decomposition, NULL/0 for the default plan).  Writes one record per
 * block in contraction order -- kind (0 leaf, 1 triangle, 2 root cycle of
 * length >= 4, 3 root node, 4 non-root cycle of length >= 4), L, L nodes,
 * number of boundary nodes, the boundary nodes, the number of children, the
 * children's block indices -- into out[cap] and aut(Q) into *aut.  Returns the
 * number of int32 words (more than cap means truncated) or a CC_ERR_ code.
 * A plan the kernels cannot run is returned too (cc_plan_supported tells). */
int cc_plan_inspect(int k, int n_edges, const int32_t *edges, const int32_t *block_seq, int seq_len,
                    int32_t *out, int cap, int64_t *aut);

/* Host-only: 1 if the kernels run the plan cc_plan_inspect describes for the
 * same arguments, 0 if not (cc_set_query / cc_set_decomposition would answer
 * CC_ERR_UNSUPPORTED), or a CC_ERR_ code for an invalid query or order.  Not
 * run: a cycle longer than 8; a cycle reading more than four Case-2 tables
 * keyed by pairs that need not be data edges (Section 4.1, Case 2: boundary
 * nodes not adjacent in their cycle); a Case-2 cycle whose longer side
 * between its boundary nodes has more than 5 edges.  (Cycles and triangles
 * that read or write such tables run on the general cycle kernel, a leaf
 * over one walks its pair graph; a root triangle that reads one has no
 * per-vertex split: cc_count_per_vertex answers CC_ERR_UNSUPPORTED for it.) */
int cc_plan_supported(int k, int n_edges, const int32_t *edges, const int32_t *block_seq, int seq_len);

/* Host-only: every decomposition tree of a query (Section 5.3), one record
 * per distinct tree -- sequence length m, supported (1 when the library has
 * kernels for every block), the paper's ranking factors (longest cycle
 * block, number of boundary nodes, number of annotations, each summed over
 * the blocks), 1 when it is the tree cc_set_query picks, 1 when it is the
 * tree the paper's factors alone pick, the library's join cost (rounded),
 * then the m-word contraction sequence in cc_set_decomposition's block_seq
 * format -- into out[cap].  *n_plans (nullable) receives the number of
 * trees.  Returns the number of int32 words (more than cap means truncated)
 * or a CC_ERR_ code.
 * cc_set_query picks, among the supported trees, the least by: longest
 * cycle block (the paper's first factor), then the join cost -- per data
 * triangle (taken as three per edge) six node assignments times the product
 * of the annotating blocks' row lengths, four times that for a triangle
 * with two or more annotations, twice for an edge-keyed output; per data
 * edge of a leaf block the product of its annotating row lengths -- then
 * the paper's remaining factors (boundary nodes, annotations). */
int cc_plan_enumerate(int k, int n_edges, const int32_t *edges, int32_t *out, int cap, int *n_plans);

/* Query facts: k, aut(Q), number of blocks, longest cycle block. */
int cc_query_info(cc_ctx *ctx, int32_t query_id, int *k, int64_t *aut, int *n_blocks,
                  int *longest_cycle);

/* Colouring seed for the hash colouring above (default 1). */
int cc_set_coloring_seed(cc_ctx *ctx, uint64_t seed);
/* Explicit colours for graph_id: colors[t * n + v] in 0..k-1 for T trials,
 * v the caller's vertex id.  Counts then use trial t's row for trial t
 * (t < T).  cc_clear_colors returns to the hash colouring. */
int cc_set_colors(cc_ctx *ctx, int32_t graph_id, const uint8_t *colors, int T);
int cc_clear_colors(cc_ctx *ctx, int32_t graph_id);

/* Plain form: count colourful matches of query_id in graph_id for trials
 * first_trial .. first_trial+T-1, one colouring per pass.
 * colorful[T]: colourful match counts (uint64).  estimate[T] (nullable):
 * colorful * k^k / k! / aut(Q), the subgraph-count estimate of that trial.
 * aut (nullable): aut(Q).  On CC_ERR_OVERFLOW the overflowing trials'
 * colorful entries are UINT64_MAX and the other trials are still filled.
 * A trial's uint64 result is fixed once its count passes 2^64-1, so the
 * general root-cycle path (annotated cycles, cycles longer than 6) stops
 * its work there. */
int cc_count(cc_ctx *ctx, int32_t graph_id, int32_t query_id, int first_trial, int T,
             uint64_t *colorful, double *estimate, double *aut);

/* Batched form.  A request asks for trials first_trial .. first_trial +
 * trials - 1 of one query on one graph.  All (request, trial) passes run on
 * the device back to back with no host round trip between them; the first
 * call for a given batch also records them as a CUDA graph, and later calls
 * with the same requests (same seed and threshold) replay that graph as one
 * launch.  colorful receives the counts of all trials, request after request
 * (sum of `trials` entries, UINT64_MAX for an overflowing trial); status
 * (nullable, n_reqs entries) receives CC_OK or CC_ERR_OVERFLOW per request.
 * Counts are identical to cc_count's.  Returns CC_OK unless a request is
 * invalid or a CUDA / memory error occurs.  A plan with a Case-2 block whose
 * table is keyed by pairs that need not be data edges sizes that table on
 * the host during the pass (a device-to-host read of its length): a batch
 * holding such a plan runs its passes with those synchronisations and is
 * not recorded as a CUDA graph. */
typedef struct cc_request {
  int32_t graph_id;
  int32_t query_id;
  int32_t first_trial;
  int32_t trials;
} cc_request;
int cc_count_batch(cc_ctx *ctx, const cc_request *reqs, int n_reqs, uint64_t *colorful, int *status);
/* Whether cc_count_batch records and replays CUDA graphs (default 1). */
int cc_set_graph_capture(cc_ctx *ctx, int enable);
/* Lanes of cc_count_batch (1..4, default 2): the batch's passes are dealt
 * out round-robin to this context and lanes - 1 auxiliary contexts, each
 * with its own CUDA stream, scratch and tables and sharing this context's
 * graphs and plans, so passes of different colourings run concurrently
 * (each lane's scratch is allocated like this context's).  A batch on a
 * graph with explicit colours (cc_set_colors) uses one lane.  Counts do not
 * depend on the lanes. */
int cc_set_batch_lanes(cc_ctx *ctx, int lanes);
/* Time the root-cycle closure of query_id on graph_id for heavy-source
 * degree thresholds 64, 96, 128, 192, ..., 3072, 4096 (steps of 1.5 and 4/3,
 * up to twice the maximum degree) on one colouring, after one untimed run,
 * and keep the fastest for this (graph, query); later counts
 * use it unless cc_set_heavy_degree forces a value.  *heavy_degree
 * (nullable) receives the choice. */
int cc_autotune(cc_ctx *ctx, int32_t graph_id, int32_t query_id, int *heavy_degree);

/* Measured choice of the decomposition tree: every supported tree of
 * query_id (at most 32, in cc_plan_enumerate's order) counts one colouring
 * of graph_id after an untimed one; the fastest becomes the query's
 * decomposition (as cc_set_decomposition would set it, for every graph).
 * *chosen (nullable) receives its index among the supported trees.  Counts
 * do not depend on the tree. */
int cc_autotune_plan(cc_ctx *ctx, int32_t graph_id, int32_t query_id, int *chosen);

/* Serving loop (continuous batching).  A server holds graphs and queries
 * resident on one device and `workers` worker contexts, each with its own
 * CUDA stream and scratch.  Requests (graph, query, trials) are submitted at
 * any time; they are admitted first-in first-out whenever a worker is idle
 * and the request's table memory (the bytes of its plan's projection tables
 * on that graph, at most (|V| or |E|) * 2^k * 8 per table) fits in what the
 * budget has left (0 = no memory limit); admitted requests run concurrently
 * on the workers' streams and a finished one frees its worker and memory for
 * the next.  colorful (host, `trials` entries) must stay valid until the
 * request's result has been polled.  Results carry submit / admit / done
 * times in seconds since the server was created.  Counts equal cc_count's
 * for the same graph, query, trials and seed. */
typedef struct cc_server cc_server;
typedef struct cc_server_result {
  int64_t ticket;
  int32_t status;  /* CC_OK, CC_ERR_OVERFLOW, ... of the request's count */
  int32_t trials;
  double submit_s, admit_s, done_s;
} cc_server_result;
int cc_server_create(cc_server **out, int device, int workers, size_t memory_budget);
void cc_server_destroy(cc_server *s);
int cc_server_load_csr(cc_server *s, int64_t n, const int64_t *row_ptr, const int32_t *col, int64_t nnz,
                       int32_t *graph_id);
int cc_server_set_query(cc_server *s, int k, int n_edges, const int32_t *edges, int32_t *query_id);
int cc_server_set_coloring_seed(cc_server *s, uint64_t seed);
/* CC_ERR_OOM when the request alone exceeds the memory budget. */
int cc_server_submit(cc_server *s, int32_t graph_id, int32_t query_id, int first_trial, int trials,
                     uint64_t *colorful, int64_t *ticket);
/* Move up to cap finished results to out, waiting up to timeout_ms for one;
 * returns how many were written. */
int cc_server_poll(cc_server *s, cc_server_result *out, int cap, int timeout_ms);
int cc_server_stats(cc_server *s, int64_t *waiting, int64_t *running, size_t *bytes_in_flight);

/* One trial, and the count split by vertex: for a root cycle block the
 * colourful matches whose highest root-cycle vertex (degree order) is v;
 * for a root that is a single node, the matches mapping that node to v.
 * per_vertex[n] is indexed by the caller's vertex ids and sums to *total.
 * On CC_ERR_OVERFLOW *total is UINT64_MAX and the split is not defined (the
 * general root-cycle path stops once the count has passed 2^64-1). */
int cc_count_per_vertex(cc_ctx *ctx, int32_t graph_id, int32_t query_id, int trial,
                        uint64_t *per_vertex, uint64_t *total);

/* Structural work of one colouring of query_id on graph_id in edge-subset
 * updates (independent of the colouring): the sum, over every
 * table-building step, of the data edges it scans times the signature slots
 * of the rows it extends.  For a root cycle of length L these are, for every
 * source u (highest cycle vertex) with at least two lower neighbours and
 * both halves (floor(L/2) and ceil(L/2) hops), the edges from each level-j
 * vertex to vertices below u, times C(k-2, j-1) slots (one slot at j = 0). */
int cc_work_units(cc_ctx *ctx, int32_t graph_id, int32_t query_id, double *units);

/* The same structural work split by the plan's stages (contraction order,
 * kinds as in cc_plan_inspect: 0 leaf, 1 triangle, 2 root cycle, 3 root
 * node).  For stage i < cap: kind[i], units[i] (edge-subset updates),
 * alg_bytes[i] (the stage's algorithmic bytes: for a leaf join 8 per update
 * that gathers a table entry, 4 per directed edge for the neighbour id and
 * 8 per table entry read from the annotating node block or written; for a
 * triangle block 4 per wedge scanned and 8 per output entry; for a root
 * cycle 4 per data edge scanned; for a root node 8 per vertex) and
 * scans[8 i + j] (root cycle: data edges scanned out of level j, both halves
 * summed; 0 for other stages).  Any output may be NULL.  Returns the number
 * of stages or a CC_ERR_ code. */
int cc_work_detail(cc_ctx *ctx, int32_t graph_id, int32_t query_id, int cap, int32_t *kind, double *units,
                   double *alg_bytes, double *scans);

/* Kernel timing: when enabled, the library brackets each kernel launch with
 * CUDA events on its stream and accumulates the time per kernel name.
 * cc_get_timing copies up to `cap` names (NUL-terminated, 48 bytes each),
 * accumulated milliseconds and launch counts; returns the number of names. */
int cc_set_timing(cc_ctx *ctx, int enable);
int cc_get_timing(cc_ctx *ctx, char *names, double *ms, int64_t *launches, int cap);
int cc_reset_timing(cc_ctx *ctx);

/* Kernels this context has launched since it was created, counting the
 * library's own kernels only (not memsets, copies or the sorting library's
 * kernels used while loading a graph); a replayed batch graph adds the
 * kernels it holds.  Counting needs no timing and no synchronisation. */
int cc_kernel_launches(cc_ctx *ctx, uint64_t *launches);

/* Count without any device allocation by the library (the paper has no
 * counterpart; it is for callers that cannot let a library allocate GPU
 * memory, e.g. code that owns a fixed device arena or runs where cudaMalloc
 * is not allowed).  Counts colourful matches of the plain cycle C_L,
 * L in {4, 5, 6} (k = L colours), in a graph given by DEVICE pointers:
 * d_row_ptr[n+1] (int64) and d_col[nnz] (int32) a symmetric simple CSR whose
 * rows are sorted ascending, d_colors[n] colours in 0..L-1.  *count (host)
 * receives the count, equal to cc_count's for the same graph, colours and
 * query.  Working memory is one static device array of 64 MiB inside the
 * library, held by every GPU that loads it until the process exits; the
 * graph must fit in it: n * 112 bytes (L = 5, 6) or n * 40 bytes (L = 4)
 * plus n * 4 bytes and 256 bytes at most 64 MiB, else CC_ERR_INVALID_ARG.
 * Maximum degree must stay below 65536 (CC_ERR_INVALID_ARG otherwise);
 * unsorted rows, out-of-range ids, self-loops or colours >= L give
 * CC_ERR_BAD_GRAPH; CC_ERR_TIMEOUT when the kernel's bounded wait gave up
 * (a contribution was skipped, so no count is returned); CC_ERR_OVERFLOW
 * with *count = UINT64_MAX when the count exceeds 2^64-1.  Work is issued on
 * cuda_stream (a cudaStream_t, NULL for the legacy stream); the call
 * synchronises that stream twice and returns when the count is on the host.
 * The first call on a device looks up the array's device address with
 * cudaGetSymbolAddress; make that first call before any stream capture on
 * that device.  All calls share the one array (each call clears what it
 * uses first), so calls that overlap on the GPU -- concurrent streams or
 * threads -- race and must be serialised by the caller.  The calling
 * thread's current device is restored on return. */
int cc_count_cycle_noalloc(int device, void *cuda_stream, int L, int64_t n, const int64_t *d_row_ptr,
                           const int32_t *d_col, const uint8_t *d_colors, uint64_t *count);

const char *cc_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* CC_H */
