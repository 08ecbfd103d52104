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
// Lanes: the passes of a batch are dealt out round-robin to `batch_lanes`
// lanes -- this context and auxiliary contexts, each on its own stream with
// its own scratch and tables, sharing this context's graphs and plans -- so
// passes of different colourings run concurrently (one lane's memory-bound
// per-CTA push beside another's issue-bound pulls, the small launches of one
// filling the gaps of another).  Every lane forks from this context's stream
// and joins it again; in the captured graph the lanes are parallel branches.
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
  std::vector<std::vector<PassBuffers>> lane_bufs;  // the same for each other lane
  std::vector<int32_t> graph_of;  // graph of each request (for freeing)
  u64 *results = nullptr;         // [total trials][8] status words
  size_t total = 0;
  cudaGraphExec_t exec = nullptr;
  uint64_t kernels = 0;           // kernels one replay launches
  cudaEvent_t fork = nullptr;     // this context's stream -> the lanes
  std::vector<cudaEvent_t> join;  // each lane -> this context's stream
};

void batch_cache_clear(Ctx &c) {
  if (c.batches.empty()) return;
  cudaStreamSynchronize(c.stream);
  if (c.own_stream) cudaStreamSynchronize(c.own_stream);
  for (auto *l : c.lanes) cudaStreamSynchronize(l->c.stream);
  for (auto &kv : c.batches) {
    Ctx::BatchCache *b = kv.second;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (size_t i = 0; i < b->bufs.size(); i++) {
      auto it = c.graphs.find(b->graph_of[i]);
      if (it != c.graphs.end()) free_pass(c, it->second, b->bufs[i]);
    }
    for (size_t j = 0; j < b->lane_bufs.size() && j < c.lanes.size(); j++) {
      Ctx &x = c.lanes[j]->c;
      for (size_t i = 0; i < b->lane_bufs[j].size(); i++) {
        auto it = x.graphs.find(b->graph_of[i]);
        if (it != x.graphs.end()) free_pass(x, it->second, b->lane_bufs[j][i]);
      }
    }
    if (b->fork) cudaEventDestroy(b->fork);
    for (auto e : b->join) cudaEventDestroy(e);
    dev_free(c, b->results, b->total * 8 * sizeof(u64));
    delete b;
  }
  c.batches.clear();
}

// The other lanes of a batch: created on first use, then brought up to date
// with this context (graphs shared, never owned; plans, seed and settings
// copied).  Returns the number of lanes usable for these requests.
static int ready_lanes(Ctx &c, const cc_request *reqs, int n) {
  int want = std::max(1, c.batch_lanes);
  for (int i = 0; i < n; i++)
    if (c.graphs[reqs[i].graph_id].colors) want = 1;  // explicit colours stay with this context
  while ((int)c.lanes.size() < want - 1) {
    cc_ctx *x = nullptr;
    if (cc_create(&x, c.device, nullptr) != CC_OK) break;
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      cc_destroy(x);
      break;
    }
    x->c.stream = x->c.own_stream = st;
    c.lanes.push_back(x);
  }
  const int lanes = std::min<int>(want, (int)c.lanes.size() + 1);
  for (int j = 0; j < lanes - 1; j++) {
    Ctx &x = c.lanes[j]->c;
    x.budget = c.budget;
    x.seed = c.seed;
    x.heavy_degree = c.heavy_degree;
    x.procedure = c.procedure;
    x.tri_list = c.tri_list;
    x.plans = c.plans;
    for (auto &kv : c.graphs) {
      DevGraph copy = kv.second;
      copy.owned = false;
      copy.colors = nullptr;
      copy.colors_T = 0;
      auto it = x.graphs.find(kv.first);
      if (it != x.graphs.end() && copy.h_push_work.empty()) copy.h_push_work = it->second.h_push_work;
      x.graphs[kv.first] = copy;
    }
    for (auto it = x.graphs.begin(); it != x.graphs.end();)
      it = c.graphs.count(it->first) ? std::next(it) : x.graphs.erase(it);
  }
  return lanes;
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

// enqueue every (request, trial) pass of the batch: pass number p goes to
// lane p mod lanes; the lanes fork from c.stream and join it at the end
static int enqueue_batch(Ctx &c, const cc_request *reqs, int n, Ctx::BatchCache &b) {
  const int lanes = (int)b.lane_bufs.size() + 1;
  if (lanes > 1) {
    if (cudaEventRecord(b.fork, c.stream) != cudaSuccess) return CC_ERR_CUDA;
    for (int j = 0; j < lanes - 1; j++)
      if (cudaStreamWaitEvent(c.lanes[j]->c.stream, b.fork, 0) != cudaSuccess) return CC_ERR_CUDA;
  }
  std::vector<uint64_t> k0(lanes - 1);
  for (int j = 0; j < lanes - 1; j++) k0[j] = c.lanes[j]->c.kernels;
  size_t slot = 0;
  for (int i = 0; i < n; i++) {
    for (int t = 0; t < reqs[i].trials; t++, slot++) {
      const int j = (int)(slot % lanes);
      Ctx &x = j == 0 ? c : c.lanes[j - 1]->c;
      PassBuffers &bufs = j == 0 ? b.bufs[i] : b.lane_bufs[j - 1][i];
      DevGraph &g = x.graphs[reqs[i].graph_id];
      Plan &p = x.plans[reqs[i].query_id];
      x.cur_tuned_heavy = g.tuned_heavy.count(reqs[i].query_id) ? g.tuned_heavy[reqs[i].query_id] : -1;
      int rc = enqueue_pass(x, g, p, (int64_t)reqs[i].first_trial + t, bufs, b.results + slot * 8, nullptr, nullptr);
      if (rc != CC_OK) return rc;
    }
  }
  for (int j = 0; j < lanes - 1; j++) {
    Ctx &x = c.lanes[j]->c;
    c.kernels += x.kernels - k0[j];
    x.kernels = k0[j];
    if (cudaEventRecord(b.join[j], x.stream) != cudaSuccess ||
        cudaStreamWaitEvent(c.stream, b.join[j], 0) != cudaSuccess)
      return CC_ERR_CUDA;
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
    // more lanes than passes would idle
    const int lanes = std::min<int>(ready_lanes(c, reqs, n_reqs), (int)std::max<size_t>(total, 1));
    b->lane_bufs.resize(lanes - 1);
    if (lanes > 1 && cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) rc = CC_ERR_CUDA;
    for (int j = 0; j < lanes - 1 && rc == CC_OK; j++) {
      b->join.push_back(nullptr);
      if (cudaEventCreateWithFlags(&b->join.back(), cudaEventDisableTiming) != cudaSuccess) rc = CC_ERR_CUDA;
    }
    for (int i = 0; i < n_reqs && rc == CC_OK; i++) {
      b->bufs.emplace_back();
      b->graph_of.push_back(reqs[i].graph_id);
      rc = alloc_pass(c, c.graphs[reqs[i].graph_id], c.plans[reqs[i].query_id], b->bufs.back());
      for (int j = 0; j < lanes - 1 && rc == CC_OK; j++) {
        Ctx &x = c.lanes[j]->c;
        b->lane_bufs[j].emplace_back();
        rc = alloc_pass(x, x.graphs[reqs[i].graph_id], x.plans[reqs[i].query_id], b->lane_bufs[j].back());
      }
    }
    // eager run: sizes the scratch and gives this call's results
    if (rc == CC_OK) rc = enqueue_batch(c, reqs, n_reqs, *b);
    // a pass with a pair-keyed block sizes its pair list on the host: not capturable
    bool host_sized = false;
    for (int i = 0; i < n_reqs; i++)
      for (auto &st : c.plans[reqs[i].query_id].stages) host_sized = host_sized || st.pair_out;
    if (rc == CC_OK && c.capture && !host_sized) {
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

extern "C" int cc_set_batch_lanes(cc_ctx *ctx, int lanes) {
  if (!ctx || lanes < 1 || lanes > 4) return CC_ERR_INVALID_ARG;
  if (ctx->c.batch_lanes != lanes) batch_cache_clear(ctx->c);
  ctx->c.batch_lanes = lanes;
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

// Measured choice of the decomposition tree (the exhaustive evaluation of
// Section "Evaluation of Plan Generation Heuristic", run on the caller's
// graph): every supported tree of the query (at most 32) counts one
// colouring after an untimed one, timed with CUDA events; the fastest becomes
// the query's decomposition.  *chosen receives its index among the supported
// trees in cc_plan_enumerate's order.
extern "C" int cc_autotune_plan(cc_ctx *ctx, int32_t graph_id, int32_t query_id, int *chosen) {
  if (!ctx) return CC_ERR_INVALID_ARG;
  Ctx &c = ctx->c;
  auto gi = c.graphs.find(graph_id);
  auto pi = c.plans.find(query_id);
  if (gi == c.graphs.end() || pi == c.plans.end()) return CC_ERR_INVALID_ARG;
  DevGraph &g = gi->second;
  const Plan orig = pi->second;
  std::vector<PlanChoice> trees;
  int rc = plan_enumerate(orig.k, orig.edges, trees);
  if (rc != CC_OK) return rc;
  std::vector<Plan> plans;
  for (auto &t : trees) {
    if (!t.supported || plans.size() >= 32) continue;
    Plan p;
    if (plan_explicit(orig.k, orig.edges, t.seq, p) == CC_OK) plans.push_back(p);
  }
  if (plans.empty()) return CC_ERR_UNSUPPORTED;
  cudaSetDevice(c.device);
  int best = 0;
  if (plans.size() > 1) {
    const bool timing = c.timing;
    c.timing = false;
    c.cur_tuned_heavy = g.tuned_heavy.count(query_id) ? g.tuned_heavy[query_id] : -1;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best_ms = 0.f;
    for (size_t i = 0; i < plans.size() && rc == CC_OK; i++) {
      u64 cnt = 0;
      bool ovf = false;
      rc = prepare_plan_graph(c, g, plans[i]);
      if (rc == CC_OK) rc = run_plan(c, g, plans[i], 1, &cnt, &ovf, nullptr, nullptr);  // untimed
      cudaEventRecord(a, c.stream);
      if (rc == CC_OK) rc = run_plan(c, g, plans[i], 0, &cnt, &ovf, nullptr, nullptr);
      cudaEventRecord(b, c.stream);
      cudaEventSynchronize(b);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      if (i == 0 || ms < best_ms) {
        best_ms = ms;
        best = (int)i;
      }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    c.timing = timing;
    if (rc != CC_OK) return rc;
  }
  pi->second = plans[best];
  for (auto &kv : c.graphs) kv.second.work_detail.erase(query_id);
  batch_cache_clear(c);
  if (chosen) *chosen = best;
  return CC_OK;
}
