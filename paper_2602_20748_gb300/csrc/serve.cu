// Serving loop: continuous batching of mixed RPQ / CRPQ requests over one
// resident graph.
//
// Requests are queued by kind.  Two worker threads, each with its own
// context (own CUDA stream, persistent grids sized to half of the SMs), run
// concurrently so their work overlaps on the device:
//   * the single-source worker takes every waiting single-source request it
//     can admit -- up to max_batch, and only while the visited bitmaps of the
//     admitted queries (states x |V| bits each) fit its memory share -- and
//     evaluates them in one batched launch (run_rpq_batch's engine).  Requests
//     that arrive while a batch is on the device join the next batch: a slot
//     opens as soon as the running batch finishes.
//   * the bulk worker takes all-pairs and CRPQ requests one at a time, oldest
//     first; an all-pairs request is one evaluation over every start vertex
//     (launches of 4,096), which a cancel stops before its next launch.
// Every request gets its row count and row digest, as the standalone call
// would report them, and its queueing / service / total latency.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "batch.h"
#include "crpq.h"
#include "rpq_internal.h"

using Clock = std::chrono::steady_clock;

namespace {

struct Req {
  uint64_t ticket = 0;
  uint32_t kind = 0;
  const rpq_query *q = nullptr;
  uint32_t source = 0;
  uint32_t n_vars = 0;
  std::vector<int32_t> var_label;
  std::vector<crpq_atom> atoms;
  Clock::time_point t_submit, t_start, t_done;
  bool done = false;
  int status = RPQ_OK;
  uint64_t count = 0, dsum = 0, dxor = 0;
};

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

struct rpq_server {
  rpq_ctx *owner = nullptr;
  rpq_ctx *ctx_single = nullptr;
  rpq_ctx *ctx_bulk = nullptr;
  cudaStream_t st_single = nullptr, st_bulk = nullptr;
  const rpq_graph *g = nullptr;
  uint64_t single_budget = 0;
  uint32_t max_batch = 4096;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req *> singles, bulk;
  std::map<uint64_t, std::unique_ptr<Req>> reqs;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::atomic<uint64_t> cancel_upto{0};  // tickets <= this are cancelled
  std::thread t_single, t_bulk;
  std::atomic<uint64_t> batches{0}, batched_requests{0};
};

namespace {

void single_worker(rpq_server *s) {
  const rpq::DevGraph &dg = rpq::graph_dev(s->g);
  const uint64_t state_bytes = ((uint64_t)dg.n + 63) / 64 * 8;
  for (;;) {
    std::vector<Req *> take;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return s->stop || !s->singles.empty(); });
      if (s->stop && s->singles.empty()) return;
      uint64_t mem = 0;
      while (!s->singles.empty() && take.size() < s->max_batch) {
        Req *r = s->singles.front();
        uint64_t need = (uint64_t)rpq::query_host(r->q).d.n_states * state_bytes;
        if (!take.empty() && mem + need > s->single_budget) break;  // admission by memory
        mem += need;
        take.push_back(r);
        s->singles.pop_front();
      }
    }
    const auto t0 = Clock::now();
    std::vector<const rpq_query *> qs;
    std::vector<uint32_t> srcs;
    for (Req *r : take) {
      qs.push_back(r->q);
      srcs.push_back(r->source);
      r->t_start = t0;
    }
    rpq::BatchOut bo;
    bo.per_query = true;
    rpq::BatchTuning tun = rpq::ctx_batch_tuning(s->ctx_single);
    tun.queries_per_launch = (uint32_t)take.size();
    int rc = rpq::batch_run(s->ctx_single, s->g, (uint32_t)take.size(), qs.data(), srcs.data(), false, tun, &bo);
    const auto t1 = Clock::now();
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (size_t i = 0; i < take.size(); i++) {
        Req *r = take[i];
        r->status = rc;
        if (rc == RPQ_OK && bo.qstats.size() >= 3 * (i + 1)) {
          r->count = bo.qstats[3 * i];
          r->dsum = bo.qstats[3 * i + 1];
          r->dxor = bo.qstats[3 * i + 2];
        }
        r->t_done = t1;
        r->done = true;
      }
      s->batches++;
      s->batched_requests += take.size();
    }
    s->cv_done.notify_all();
  }
}

void bulk_worker(rpq_server *s) {
  for (;;) {
    Req *r = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return s->stop || !s->bulk.empty(); });
      if (s->stop && s->bulk.empty()) return;
      r = s->bulk.front();
      s->bulk.pop_front();
      rpq::ctx_set_cancel(s->ctx_bulk, false);
    }
    r->t_start = Clock::now();
    int rc = RPQ_OK;
    uint64_t count = 0, dsum = 0, dxor = 0;
    if (r->kind == RPQ_REQ_ALLPAIRS) {
      // one all-pairs evaluation (start vertices without a usable edge are
      // dropped up front; the rest run in full launches); a cancel stops it
      // before its next launch
      rpq_result *res = nullptr;
      rc = run_rpq(s->ctx_bulk, s->g, r->q, nullptr, 0, RPQ_COUNT_ONLY, &res);
      if (rc == RPQ_OK) {
        result_info(res, &count, nullptr, &dsum, &dxor);
        free_result(res);
      }
    } else {
      rpq_result *res = nullptr;
      rc = run_crpq(s->ctx_bulk, s->g, r->n_vars, r->var_label.empty() ? nullptr : r->var_label.data(),
                    r->atoms.data(), (uint32_t)r->atoms.size(), nullptr, 0, RPQ_COUNT_ONLY, &res);
      if (rc == RPQ_OK) {
        result_info(res, &count, nullptr, &dsum, &dxor);
        free_result(res);
      }
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      r->status = rc;
      r->count = count;
      r->dsum = dsum;
      r->dxor = dxor;
      r->t_done = Clock::now();
      r->done = true;
    }
    s->cv_done.notify_all();
  }
}

}  // namespace

extern "C" {

int rpq_server_create(rpq_ctx *ctx, const rpq_graph *g, uint64_t mem_budget_bytes, uint32_t max_batch,
                      rpq_server **out) {
  if (!ctx || !g || !out || max_batch == 0) return rpq::ctx_error(ctx, RPQ_ERR_INVALID_ARG, "bad argument");
  *out = nullptr;
  const int dev = rpq::ctx_device(ctx);
  if (dev < 0) return rpq::ctx_error(ctx, RPQ_ERR_NO_DEVICE, "host-only context has no GPU");
  cudaSetDevice(dev);
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  uint64_t budget = mem_budget_bytes ? mem_budget_bytes : (uint64_t)(free_b * 0.8);
  auto *s = new rpq_server;
  s->owner = ctx;
  s->g = g;
  s->max_batch = max_batch;
  if (cudaStreamCreateWithFlags(&s->st_single, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->st_bulk, cudaStreamNonBlocking) != cudaSuccess) {
    delete s;
    return rpq::ctx_error(ctx, RPQ_ERR_CUDA, "stream creation failed");
  }
  int rc = rpq_create(&s->ctx_single, dev, budget / 2, s->st_single);
  if (rc == RPQ_OK) rc = rpq_create(&s->ctx_bulk, dev, budget / 2, s->st_bulk);
  if (rc != RPQ_OK) {
    rpq_destroy(s->ctx_single);
    cudaStreamDestroy(s->st_single);
    cudaStreamDestroy(s->st_bulk);
    delete s;
    return rpq::ctx_error(ctx, rc, "worker context creation failed");
  }
  // the workers follow the owner's tunables and share the device: half of
  // the SMs each for persistent grids
  rpq::ctx_copy_tunables(s->ctx_single, ctx);
  rpq::ctx_copy_tunables(s->ctx_bulk, ctx);
  rpq_set_option(s->ctx_single, "grid_share", 0.5);
  rpq_set_option(s->ctx_bulk, "grid_share", 0.5);
  // visited bitmaps get a third of the single worker's share; the rest holds
  // frontier lists and results
  s->single_budget = budget / 6;
  s->t_single = std::thread(single_worker, s);
  s->t_bulk = std::thread(bulk_worker, s);
  *out = s;
  return RPQ_OK;
}

int rpq_server_submit(rpq_server *s, const rpq_request *req, uint64_t *ticket) {
  if (!s || !req || !ticket) return RPQ_ERR_INVALID_ARG;
  const rpq::DevGraph &dg = rpq::graph_dev(s->g);
  auto r = std::make_unique<Req>();
  r->kind = req->kind;
  if (req->kind == RPQ_REQ_SINGLE || req->kind == RPQ_REQ_ALLPAIRS) {
    if (!req->q) return RPQ_ERR_INVALID_ARG;
    if (req->kind == RPQ_REQ_SINGLE && req->source >= dg.n) return RPQ_ERR_INVALID_ARG;
    r->q = req->q;
    r->source = req->source;
  } else if (req->kind == RPQ_REQ_CRPQ) {
    if (!req->atoms || req->n_atoms == 0 || req->n_vars == 0) return RPQ_ERR_INVALID_ARG;
    r->n_vars = req->n_vars;
    r->atoms.assign(req->atoms, req->atoms + req->n_atoms);
    if (req->var_label) r->var_label.assign(req->var_label, req->var_label + req->n_vars);
  } else {
    return RPQ_ERR_INVALID_ARG;
  }
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return RPQ_ERR_INVALID_ARG;
    r->ticket = s->next_ticket++;
    *ticket = r->ticket;
    Req *raw = r.get();
    s->reqs[r->ticket] = std::move(r);
    if (raw->kind == RPQ_REQ_SINGLE)
      s->singles.push_back(raw);
    else
      s->bulk.push_back(raw);
  }
  s->cv_work.notify_all();
  return RPQ_OK;
}

int rpq_server_wait(rpq_server *s, uint64_t ticket, double timeout_s, rpq_reply *reply) {
  if (!s || !reply) return RPQ_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return RPQ_ERR_INVALID_ARG;
  Req *r = it->second.get();
  auto pred = [&] { return r->done; };
  if (timeout_s < 0)
    s->cv_done.wait(lk, pred);
  else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred))
    return RPQ_ERR_TIMEOUT;
  reply->status = r->status;
  reply->count = r->count;
  reply->digest_sum = r->dsum;
  reply->digest_xor = r->dxor;
  reply->queued_ms = ms_between(r->t_submit, r->t_start);
  reply->service_ms = ms_between(r->t_start, r->t_done);
  reply->latency_ms = ms_between(r->t_submit, r->t_done);
  s->reqs.erase(it);
  return RPQ_OK;
}

int rpq_server_cancel(rpq_server *s) {
  if (!s) return RPQ_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->cancel_upto = s->next_ticket - 1;
    rpq::ctx_set_cancel(s->ctx_bulk, true);  // the bulk request in service, if any
    const auto now = Clock::now();
    for (auto *q : {&s->singles, &s->bulk}) {
      for (Req *r : *q) {
        r->status = RPQ_ERR_CANCELLED;
        r->t_start = r->t_done = now;
        r->done = true;
      }
      q->clear();
    }
  }
  s->cv_done.notify_all();
  return RPQ_OK;
}

int rpq_server_stats(rpq_server *s, uint64_t *batches, uint64_t *batched_requests) {
  if (!s) return RPQ_ERR_INVALID_ARG;
  if (batches) *batches = s->batches;
  if (batched_requests) *batched_requests = s->batched_requests;
  return RPQ_OK;
}

void rpq_server_destroy(rpq_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->t_single.joinable()) s->t_single.join();
  if (s->t_bulk.joinable()) s->t_bulk.join();
  rpq_destroy(s->ctx_single);
  rpq_destroy(s->ctx_bulk);
  cudaStreamDestroy(s->st_single);
  cudaStreamDestroy(s->st_bulk);
  delete s;
}

}  // extern "C"
