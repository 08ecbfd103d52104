// Batched form and the heavy-threshold autotuner.
//
// A batch is a list of (graph, query, first trial, trials) requests.  Every
// (request, trial) colouring pass is enqueued back to back on one stream --
// colours, block tables, root reduction, status words into a per-trial slot
// -- with no host synchronisation between passes, and the whole sequence is
// captured once into a CUDA graph.  Repeating the same batch replays the
// instantiated graph: one launch for all passes, no per-pass host work.  The
// kernels leave their scratch zeroed, so a replay needs no clearing.
//
// The autotuner times the root-cycle closure for a few heavy/light degree
// thresholds on one colouring and keeps the fastest for the (graph, query).
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "cc_kernels.h"

namespace cc {

struct Ctx::BatchCache {
  std::vector<PassBuffers> bufs;  // one per request (its trials reuse them in order)
  std::vector<int32_t> graph_of;  // graph of each request (for freeing)
  u64 *results = nullptr;         // [total trials][8] status words
  size_t total = 0;
  cudaGraphExec_t exec = nullptr;
  uint64_t kernels = 0;           // kernels one replay launches
};

void batch_cache_clear(Ctx &c) {
  if (c.batches.empty()) return;
  cudaStreamSynchronize(c.stream);
  if (c.own_stream) cudaStreamSynchronize(c.own_stream);
  for (auto &kv : c.batches) {
    Ctx::BatchCache *b = kv.second;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (size_t i = 0; i < b->bufs.size(); i++) {
      auto it = c.graphs.find(b->graph_of[i]);
      if (it != c.graphs.end()) free_pass(c, it->second, b->bufs[i]);
    }
    dev_free(c, b->results, b->total * 8 * sizeof(u64));
    delete b;
  }
  c.batches.clear();
}

}  // namespace cc

using namespace cc;

static std::string batch_key(const Ctx &c, const cc_request *reqs, int n) {
  std::string k;
  for (int i = 0; i < n; i++) {
    const cc_request &r = reqs[i];
    k += std::to_string(r.graph_id) + ":" + std::to_string(r.query_id) + ":" + std::to_string(r.first_trial) +
         ":" + std::to_string(r.trials) + ";";
  }
  k += "|" + std::to_string(c.heavy_degree) + "|" + std::to_string(c.seed);
  return k;
}

// enqueue every (request, trial) pass of the batch on c.stream
static int enqueue_batch(Ctx &c, const cc_request *reqs, int n, Ctx::BatchCache &b) {
  size_t slot = 0;
  for (int i = 0; i < n; i++) {
    DevGraph &g = c.graphs[reqs[i].graph_id];
    Plan &p = c.plans[reqs[i].query_id];
    c.cur_tuned_heavy = g.tuned_heavy.count(reqs[i].query_id) ? g.tuned_heavy[reqs[i].query_id] : -1;
    for (int t = 0; t < reqs[i].trials; t++, slot++) {
      int rc = enqueue_pass(c, g, p, (int64_t)reqs[i].first_trial + t, b.bufs[i], b.results + slot * 8, nullptr,
                            nullptr);
      if (rc != CC_OK) return rc;
    }
  }
  return CC_OK;
}

extern "C" int cc_count_batch(cc_ctx *ctx, const cc_request *reqs, int n_reqs, uint64_t *colorful, int *status) {
  if (!ctx || !reqs || n_reqs <= 0 || !colorful) return CC_ERR_INVALID_ARG;
  Ctx &c = ctx->c;
  cudaSetDevice(c.device);
  size_t total = 0;
  for (int i = 0; i < n_reqs; i++) {
    const cc_request &r = reqs[i];
    auto gi = c.graphs.find(r.graph_id);
    auto pi = c.plans.find(r.query_id);
    if (gi == c.graphs.end() || pi == c.plans.end() || r.trials <= 0 || r.first_trial < 0) return CC_ERR_INVALID_ARG;
    if (!pi->second.supported) return CC_ERR_UNSUPPORTED;
    if (gi->second.colors && (gi->second.colors_max >= pi->second.k ||
                              r.first_trial + r.trials > gi->second.colors_T))
      return CC_ERR_INVALID_ARG;
    total += (size_t)r.trials;
  }
  // colouring-independent structure first (it synchronises: not under capture)
  for (int i = 0; i < n_reqs; i++) {
    int rc0 = prepare_plan_graph(c, c.graphs[reqs[i].graph_id], c.plans[reqs[i].query_id]);
    if (rc0 != CC_OK) return rc0;
  }
  // capture needs a stream other than the legacy default one
  cudaStream_t user = c.stream;
  if (!c.own_stream && cudaStreamCreateWithFlags(&c.own_stream, cudaStreamNonBlocking) != cudaSuccess)
    return CC_ERR_CUDA;
  cudaEvent_t ev;
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return CC_ERR_CUDA;
  cudaEventRecord(ev, user);
  cudaStreamWaitEvent(c.own_stream, ev, 0);
  c.stream = c.own_stream;
  const bool timing = c.timing;
  int rc = CC_OK;
  std::string key = batch_key(c, reqs, n_reqs);
  Ctx::BatchCache *b = nullptr;
  auto it = c.batches.find(key);
  if (it != c.batches.end() && it->second->exec && !c.scratch_dirty && !c.hv_dirty) {
    b = it->second;
    timing_begin(c, "batch_graph");
    rc = cudaGraphLaunch(b->exec, c.stream) == cudaSuccess ? CC_OK : CC_ERR_CUDA;
    if (rc == CC_OK) c.kernels += b->kernels;
    timing_end(c);
  } else {
    // a stale entry, or too many distinct batches held: start the cache afresh
    if (it != c.batches.end() || c.batches.size() >= 8) batch_cache_clear(c);
    b = new Ctx::BatchCache();
    b->total = total;
    b->results = (u64 *)dev_alloc(c, total * 8 * sizeof(u64));
    if (!b->results) rc = CC_ERR_OOM;
    for (int i = 0; i < n_reqs && rc == CC_OK; i++) {
      b->bufs.emplace_back();
      b->graph_of.push_back(reqs[i].graph_id);
      rc = alloc_pass(c, c.graphs[reqs[i].graph_id], c.plans[reqs[i].query_id], b->bufs.back());
    }
    // eager run: sizes the scratch and gives this call's results
    if (rc == CC_OK) rc = enqueue_batch(c, reqs, n_reqs, *b);
    if (rc == CC_OK && c.capture) {
      // record the same sequence as a CUDA graph for later replays
      if (cudaStreamSynchronize(c.stream) != cudaSuccess) rc = CC_ERR_CUDA;
      c.timing = false;
      cudaGraph_t graph = nullptr;
      if (rc == CC_OK && cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        const uint64_t k0 = c.kernels;
        int rc2 = enqueue_batch(c, reqs, n_reqs, *b);
        b->kernels = c.kernels - k0;  // recorded, not launched
        c.kernels = k0;
        cudaError_t e = cudaStreamEndCapture(c.stream, &graph);
        if (rc2 == CC_OK && e == cudaSuccess && graph &&
            cudaGraphInstantiate(&b->exec, graph, 0) == cudaSuccess) {
          // captured
        } else {
          b->exec = nullptr;
        }
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
      }
      c.timing = timing;
    }
    c.batches[key] = b;
  }
  std::vector<u64> res(total * 8, 0);
  if (rc == CC_OK &&
      (cudaMemcpyAsync(res.data(), b->results, total * 8 * sizeof(u64), cudaMemcpyDeviceToHost, c.stream) !=
           cudaSuccess ||
       cudaStreamSynchronize(c.stream) != cudaSuccess))
    rc = CC_ERR_CUDA;
  timing_flush(c);
  c.stream = user;
  cudaEventDestroy(ev);
  if (rc != CC_OK) {
    c.scratch_dirty = c.hv_dirty = true;
    batch_cache_clear(c);
    return rc;
  }
  size_t slot = 0;
  for (int i = 0; i < n_reqs; i++) {
    int st = CC_OK;
    for (int t = 0; t < reqs[i].trials; t++, slot++) {
      int sc = status_code(&res[slot * 8]);
      colorful[slot] = sc == CC_ERR_OVERFLOW ? UINT64_MAX : res[slot * 8 + ST_COUNT];
      if (sc != CC_OK && st == CC_OK) st = sc;
    }
    if (status) status[i] = st;
  }
  return CC_OK;
}

extern "C" int cc_set_graph_capture(cc_ctx *ctx, int enable) {
  if (!ctx) return CC_ERR_INVALID_ARG;
  ctx->c.capture = enable != 0;
  if (!enable) batch_cache_clear(ctx->c);
  return CC_OK;
}

extern "C" int cc_autotune(cc_ctx *ctx, int32_t graph_id, int32_t query_id, int *heavy_degree) {
  if (!ctx) return CC_ERR_INVALID_ARG;
  Ctx &c = ctx->c;
  auto gi = c.graphs.find(graph_id);
  auto pi = c.plans.find(query_id);
  if (gi == c.graphs.end() || pi == c.plans.end()) return CC_ERR_INVALID_ARG;
  if (!pi->second.supported) return CC_ERR_UNSUPPORTED;
  DevGraph &g = gi->second;
  Plan &p = pi->second;
  bool has_cycle = false;
  for (auto &st : p.stages) has_cycle = has_cycle || st.kind == ST_CYCLE_ROOT;
  cudaSetDevice(c.device);
  int best = 256;
  if (has_cycle && g.max_deg > 0) {
    const int saved = c.heavy_degree;
    const bool timing = c.timing;
    c.timing = false;
    float best_ms = 0.f;
    bool first = true;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    // thresholds 64 .. 4096 in steps of 1.5 and 4/3; one untimed run first
    // takes the one-time costs (scratch allocation, per-graph tables)
    static const int kCandidates[] = {64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048, 3072, 4096};
    {
      u64 cnt = 0;
      bool ovf = false;
      c.heavy_degree = 256;
      int rc = run_plan(c, g, p, 0, &cnt, &ovf, nullptr, nullptr);
      if (rc == CC_OK && cudaStreamSynchronize(c.stream) != cudaSuccess) rc = CC_ERR_CUDA;
      if (rc != CC_OK) {
        c.heavy_degree = saved;
        c.timing = timing;
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        return rc;
      }
    }
    for (int hd : kCandidates) {
      if (hd > 2 * g.max_deg && !first) break;
      c.heavy_degree = hd;
      u64 cnt = 0;
      bool ovf = false;
      cudaEventRecord(a, c.stream);
      int rc = run_plan(c, g, p, 0, &cnt, &ovf, nullptr, nullptr);
      cudaEventRecord(b, c.stream);
      cudaEventSynchronize(b);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      if (rc != CC_OK) {
        c.heavy_degree = saved;
        c.timing = timing;
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        return rc;
      }
      if (first || ms < best_ms) {
        best_ms = ms;
        best = hd;
      }
      first = false;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    c.heavy_degree = saved;
    c.timing = timing;
  }
  g.tuned_heavy[query_id] = best;
  batch_cache_clear(c);
  if (heavy_degree) *heavy_degree = best;
  return CC_OK;
}
