// Serving loop: continuous batching of count requests over resident graphs.
//
// A server owns one loading context (graphs, queries) and W worker contexts,
// each with its own CUDA stream and scratch, that share the loaded graphs.
// Requests arrive at any time (cc_server_submit).  The dispatcher admits
// them first-in first-out whenever a worker is idle and the request's table
// memory fits in what the budget has left; an admitted request runs on a
// worker's stream while others run on theirs, so the work of different
// requests overlaps on the device.  A finished request frees its worker and
// its memory, which admits the next waiting ones.  Every result carries its
// submit, admit and completion times.
//
// Admission cost of a request: the bytes of the projection tables its plan
// holds at once on its graph (dense rows, see the executor), plus the
// colouring buffer -- never more than (|V| or |E|) x 2^k x 8 bytes per table
// for the signature-indexed tables a k-node query needs.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "cc_kernels.h"

struct ServeReq {
  int64_t ticket;
  int32_t graph_id, query_id;
  int first_trial, trials;
  uint64_t *out;
  size_t bytes;
  double t_submit = 0, t_admit = 0, t_done = 0;
  int status = 0;
};

struct cc_server {
  int device = 0;
  cc_ctx *owner = nullptr;
  std::vector<cc_ctx *> workers;
  std::vector<std::thread> threads;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<ServeReq *> pending, admitted, done;
  size_t budget = 0, in_flight = 0;
  int idle = 0, running = 0;
  bool stop = false;
  int64_t next_ticket = 1;
  std::chrono::steady_clock::time_point t0;
  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

// admit from the head of the queue while a worker is idle and memory fits
void admit_locked(cc_server *s) {
  while (!s->pending.empty() && s->idle > (int)s->admitted.size()) {
    ServeReq *r = s->pending.front();
    if (s->budget && s->in_flight + r->bytes > s->budget && s->in_flight > 0) break;
    s->pending.pop_front();
    s->in_flight += r->bytes;
    r->t_admit = s->now();
    s->admitted.push_back(r);
    s->cv_work.notify_one();
  }
}

void worker_loop(cc_server *s, int wi) {
  cc_ctx *w = s->workers[wi];
  cudaSetDevice(s->device);
  while (true) {
    ServeReq *r = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return s->stop || !s->admitted.empty(); });
      if (s->stop && s->admitted.empty()) return;
      r = s->admitted.front();
      s->admitted.pop_front();
      s->idle--;
      s->running++;
    }
    int rc = cc_count(w, r->graph_id, r->query_id, r->first_trial, r->trials, r->out, nullptr, nullptr);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      r->status = rc;
      r->t_done = s->now();
      s->in_flight -= r->bytes;
      s->idle++;
      s->running--;
      s->done.push_back(r);
      admit_locked(s);
    }
    s->cv_done.notify_all();
  }
}

}  // namespace

using namespace cc;

extern "C" int cc_server_create(cc_server **out, int device, int workers, size_t memory_budget) {
  if (!out || workers < 1 || workers > 64) return CC_ERR_INVALID_ARG;
  *out = nullptr;
  cc_server *s = new cc_server();
  s->device = device;
  s->budget = memory_budget;
  s->t0 = std::chrono::steady_clock::now();
  int rc = cc_create(&s->owner, device, nullptr);
  for (int i = 0; i < workers && rc == CC_OK; i++) {
    cudaSetDevice(device);
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      rc = CC_ERR_CUDA;
      break;
    }
    cc_ctx *w = nullptr;
    rc = cc_create(&w, device, st);
    if (rc == CC_OK) {
      w->c.own_stream = st;  // destroyed with the worker context
      s->workers.push_back(w);
    } else {
      cudaStreamDestroy(st);
    }
  }
  if (rc != CC_OK) {
    for (auto *w : s->workers) cc_destroy(w);
    if (s->owner) cc_destroy(s->owner);
    delete s;
    return rc;
  }
  s->idle = workers;
  for (int i = 0; i < workers; i++) s->threads.emplace_back(worker_loop, s, i);
  *out = s;
  return CC_OK;
}

extern "C" void cc_server_destroy(cc_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto &t : s->threads) t.join();
  for (auto *r : s->pending) delete r;
  for (auto *r : s->admitted) delete r;
  for (auto *r : s->done) delete r;
  // workers hold borrowed graphs: release them before the owner frees the arrays
  for (auto *w : s->workers) cc_destroy(w);
  cc_destroy(s->owner);
  delete s;
}

extern "C" int cc_server_load_csr(cc_server *s, int64_t n, const int64_t *row_ptr, const int32_t *col, int64_t nnz,
                                  int32_t *graph_id) {
  if (!s || !graph_id) return CC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  int rc = cc_load_csr(s->owner, n, row_ptr, col, nnz, graph_id);
  if (rc != CC_OK) return rc;
  // the triangle list is built here, once, by the loading context: workers
  // share the graph's arrays and never build it themselves
  DevGraph &g = s->owner->c.graphs[*graph_id];
  if (s->owner->c.tri_list && (rc = tri_list_build(s->owner->c, g)) != CC_OK) return rc;
  // every worker sees the same device arrays under the same id
  for (auto *w : s->workers) {
    DevGraph b = g;
    b.owned = false;
    b.colors = nullptr;
    b.colors_T = 0;
    w->c.graphs[*graph_id] = b;
    w->c.next_graph = std::max(w->c.next_graph, *graph_id + 1);
  }
  return CC_OK;
}

extern "C" int cc_server_set_query(cc_server *s, int k, int n_edges, const int32_t *edges, int32_t *query_id) {
  if (!s || !query_id) return CC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  int rc = cc_set_query(s->owner, k, n_edges, edges, query_id);
  if (rc != CC_OK) return rc;
  for (auto *w : s->workers) {
    w->c.plans[*query_id] = s->owner->c.plans[*query_id];
    w->c.next_query = std::max(w->c.next_query, *query_id + 1);
  }
  return CC_OK;
}

extern "C" int cc_server_set_coloring_seed(cc_server *s, uint64_t seed) {
  if (!s) return CC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  cc_set_coloring_seed(s->owner, seed);
  for (auto *w : s->workers) cc_set_coloring_seed(w, seed);
  return CC_OK;
}

extern "C" int cc_server_submit(cc_server *s, int32_t graph_id, int32_t query_id, int first_trial, int trials,
                                uint64_t *colorful, int64_t *ticket) {
  if (!s || !colorful || trials <= 0 || first_trial < 0) return CC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto gi = s->owner->c.graphs.find(graph_id);
  auto pi = s->owner->c.plans.find(query_id);
  if (gi == s->owner->c.graphs.end() || pi == s->owner->c.plans.end()) return CC_ERR_INVALID_ARG;
  if (!pi->second.supported) return CC_ERR_UNSUPPORTED;
  ServeReq *r = new ServeReq();
  r->ticket = s->next_ticket++;
  r->graph_id = graph_id;
  r->query_id = query_id;
  r->first_trial = first_trial;
  r->trials = trials;
  r->out = colorful;
  r->bytes = request_table_bytes(pi->second, gi->second);
  if (s->budget && r->bytes > s->budget) {
    delete r;
    return CC_ERR_OOM;  // could never be admitted
  }
  r->t_submit = s->now();
  s->pending.push_back(r);
  if (ticket) *ticket = r->ticket;
  admit_locked(s);
  return CC_OK;
}

extern "C" int cc_server_poll(cc_server *s, cc_server_result *out, int cap, int timeout_ms) {
  if (!s || (!out && cap > 0)) return CC_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->done.empty() && timeout_ms > 0)
    s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return !s->done.empty(); });
  int n = 0;
  while (n < cap && !s->done.empty()) {
    ServeReq *r = s->done.front();
    s->done.pop_front();
    out[n].ticket = r->ticket;
    out[n].status = r->status;
    out[n].trials = r->trials;
    out[n].submit_s = r->t_submit;
    out[n].admit_s = r->t_admit;
    out[n].done_s = r->t_done;
    delete r;
    n++;
  }
  return n;
}

extern "C" int cc_server_stats(cc_server *s, int64_t *pending, int64_t *running, size_t *bytes_in_flight) {
  if (!s) return CC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (pending) *pending = (int64_t)(s->pending.size() + s->admitted.size());
  if (running) *running = s->running;
  if (bytes_in_flight) *bytes_in_flight = s->in_flight;
  return CC_OK;
}
