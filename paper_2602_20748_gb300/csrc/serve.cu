// Serving loop: continuous batching of mixed RPQ / CRPQ requests over one
// resident graph.
//
// Single-source requests go into a ring in mapped host memory that a
// persistent serving launch (batch.cu, serve_kernel) reads at every level
// boundary: a request that arrives while others are being expanded takes a
// free slot at the next level and is expanded together with them; each slot
// keeps a small open-addressing visited set and result set, and a query's
// rows are counted and digested as they are found, so its reply is ready the
// level its frontier runs empty.  The launch ends when nothing is in flight;
// the driver thread launches it again when requests arrive.  A query that
// grows past the eviction threshold leaves the launch and is evaluated by the
// lane worker, which packs every such query waiting into lane-mode launches
// of the multi-source engine (one automaton per bit lane).  All-pairs
// requests and CRPQs go to two bulk workers, each starting the oldest request
// whose device-memory estimate (traversal state, entry lists, emission
// scratch) fits what the running bulk requests leave of the bulk budget.
// The three kinds of work run on their own streams with their own shares of
// the SMs, so their launches overlap on the device.  Every request gets its
// row count and row digest, as the standalone call would report them, and its
// queueing / service / total latency.
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
#include <unordered_map>
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
  bool cancelled = false;  // a reply that still arrives is dropped
  bool waited = false;     // its reply was taken by rpq_server_wait
  int status = RPQ_OK;
  uint64_t count = 0, dsum = 0, dxor = 0;
  uint64_t reserve = 0;    // bulk: device bytes reserved while it runs
};

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

// SM shares of the three kinds of work (they sum below 1, so that the
// cooperative launches of all three fit on the device at once)
constexpr double SHARE_SERVE = 0.2, SHARE_LANE = 0.55, SHARE_BULK = 0.1;
constexpr int BULK_WORKERS = 2;
constexpr uint32_t SERVE_HASH_BITS = 13;  // 8,192-slot visited and result sets per query
constexpr uint64_t SERVE_EVICT_AT = 4096;  // product vertices before a query moves to lane mode

}  // namespace

struct rpq_server {
  rpq_ctx *owner = nullptr;
  rpq_ctx *ctx_serve = nullptr, *ctx_lane = nullptr, *ctx_bulk[BULK_WORKERS] = {nullptr, nullptr};
  cudaStream_t streams[2 + BULK_WORKERS] = {};
  const rpq_graph *g = nullptr;
  rpq::ServeEngine *eng = nullptr;
  uint32_t lanes = 4096;
  uint32_t slots = 0;
  uint64_t bulk_budget = 0, bulk_reserved = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_lane, cv_bulk, cv_done;
  std::deque<Req *> singles, lane_q, bulk;
  std::unordered_map<uint64_t, Req *> inflight;  // singles in the ring or the serving launch
  std::map<uint64_t, std::unique_ptr<Req>> reqs;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread t_single, t_lane, t_bulk[BULK_WORKERS];
  std::atomic<uint64_t> lane_launches{0}, lane_requests{0};
};

namespace {

void complete(rpq_server *s, Req *r, int status, uint64_t count, uint64_t dsum, uint64_t dxor) {
  // with s->mu held
  if (r->done) return;
  r->status = status;
  r->count = count;
  r->dsum = dsum;
  r->dxor = dxor;
  r->t_done = Clock::now();
  r->done = true;
}

// Drives the serving launch: moves waiting singles into the ring, launches
// when needed, and turns replies into completions (evicted ones go to the
// lane worker).
void single_driver(rpq_server *s) {
  cudaSetDevice(rpq::ctx_device(s->ctx_serve));
  std::vector<rpq::ServeReply> replies;
  std::vector<uint64_t> lost;
  for (;;) {
    bool idle = false;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->singles.empty() && s->inflight.empty()) {
        if (s->stop) return;
        s->cv_work.wait(lk, [&] { return s->stop || !s->singles.empty(); });
        if (s->stop && s->singles.empty() && s->inflight.empty()) return;
      }
      const auto now = Clock::now();
      while (!s->singles.empty()) {
        Req *r = s->singles.front();
        if (!rpq::serve_engine_push(s->eng, r->ticket, rpq::query_host(r->q).d, r->source)) break;
        r->t_start = now;
        s->inflight[r->ticket] = r;
        s->singles.pop_front();
      }
    }
    lost.clear();
    const int rc = rpq::serve_engine_kick(s->eng, &lost);
    replies.clear();
    rpq::serve_engine_poll(s->eng, &replies);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (const rpq::ServeReply &rp : replies) {
        auto it = s->inflight.find(rp.ticket);
        if (it == s->inflight.end()) continue;
        Req *r = it->second;
        s->inflight.erase(it);
        if (r->cancelled) {
          if (r->waited) s->reqs.erase(rp.ticket);
          continue;
        }
        if (rp.evicted) {
          s->lane_q.push_back(r);
          continue;
        }
        complete(s, r, RPQ_OK, rp.count, rp.dsum, rp.dxor);
      }
      if (rc != RPQ_OK) {
        for (uint64_t t : lost) {
          auto it = s->inflight.find(t);
          if (it == s->inflight.end()) continue;
          Req *r = it->second;
          s->inflight.erase(it);
          if (r->cancelled && r->waited) {
            s->reqs.erase(t);
            continue;
          }
          complete(s, r, rc, 0, 0, 0);
        }
      }
      idle = s->inflight.empty() && s->singles.empty();
    }
    s->cv_done.notify_all();
    s->cv_lane.notify_one();
    if (!idle) std::this_thread::sleep_for(std::chrono::microseconds(30));
  }
}

// Evaluates the queries the serving launch evicted, every one waiting at
// once, in lane-mode launches.
void lane_worker(rpq_server *s) {
  cudaSetDevice(rpq::ctx_device(s->ctx_lane));
  for (;;) {
    std::vector<Req *> take;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->stop)
        s->cv_lane.wait_for(lk, std::chrono::milliseconds(1), [&] { return !s->lane_q.empty(); });
      else
        s->cv_lane.wait(lk, [&] { return s->stop || !s->lane_q.empty(); });
      if (s->lane_q.empty()) {
        if (s->stop && s->singles.empty() && s->inflight.empty()) return;
        continue;
      }
      while (!s->lane_q.empty() && take.size() < s->lanes) {
        take.push_back(s->lane_q.front());
        s->lane_q.pop_front();
      }
    }
    std::vector<rpq::LaneTask> tasks(take.size());
    for (size_t i = 0; i < take.size(); i++) {
      tasks[i].q = take[i]->q;
      tasks[i].source = take[i]->source;
    }
    std::vector<uint64_t> ls;
    rpq_stats st{};
    const int rc = rpq::rpq_lane_stats_lanes(s->ctx_lane, s->g, tasks, s->lanes, &ls, &st);
    s->lane_launches += st.bfs_launches;
    s->lane_requests += take.size();
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (size_t i = 0; i < take.size(); i++) {
        if (take[i]->cancelled) continue;
        if (rc == RPQ_OK)
          complete(s, take[i], RPQ_OK, ls[3 * i], ls[3 * i + 1], ls[3 * i + 2]);
        else
          complete(s, take[i], rc, 0, 0, 0);
      }
    }
    s->cv_done.notify_all();
  }
}

// Device bytes an all-pairs evaluation of q with G lane groups of 256 start
// vertices holds: visited and frontier words, entry lists, claims, emission
// counts and offsets.
uint64_t allpairs_bytes(const rpq::DevGraph &g, uint32_t Q, uint32_t G) {
  const uint64_t words = (uint64_t)G * Q * g.n * 4;
  const uint64_t segs = (g.n + rpq::EMIT_SEG - 1) / rpq::EMIT_SEG;
  return words * 8 * 3 + (uint64_t)G * Q * g.n * (16 + 4) + (uint64_t)G * 256 * segs * 12 + (64ull << 20);
}

// Lane groups a bulk request runs with, and the bytes it reserves: as many
// groups (up to 16) as fit what the running bulk requests leave.
uint32_t bulk_groups(rpq_server *s, const Req *r, uint64_t *bytes) {
  const rpq::DevGraph &g = rpq::graph_dev(s->g);
  uint32_t Q = 1;
  if (r->kind == RPQ_REQ_ALLPAIRS) {
    Q = std::max(1u, rpq::query_host(r->q).d.n_states);
  } else {
    for (const crpq_atom &a : r->atoms) Q = std::max(Q, rpq::query_host(a.q).d.n_states);
  }
  const uint64_t free_b = s->bulk_budget > s->bulk_reserved ? s->bulk_budget - s->bulk_reserved : 0;
  for (uint32_t G = 16; G >= 1; G /= 2) {
    const uint64_t b = allpairs_bytes(g, Q, G) * (r->kind == RPQ_REQ_CRPQ ? 2 : 1);
    if (b <= free_b) {
      *bytes = b;
      return G;
    }
  }
  *bytes = allpairs_bytes(g, Q, 1) * (r->kind == RPQ_REQ_CRPQ ? 2 : 1);
  return 0;  // does not fit now
}

void bulk_worker(rpq_server *s, int w) {
  rpq_ctx *ctx = s->ctx_bulk[w];
  cudaSetDevice(rpq::ctx_device(ctx));
  for (;;) {
    Req *r = nullptr;
    uint32_t G = 0;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (;;) {
        if (s->stop && s->bulk.empty()) return;
        if (!s->bulk.empty()) {
          uint64_t bytes = 0;
          G = bulk_groups(s, s->bulk.front(), &bytes);
          // admission by memory: the oldest request starts once its estimate
          // fits; one that could never fit runs alone with the whole budget
          if (G == 0 && s->bulk_reserved == 0) G = 1;
          if (G) {
            r = s->bulk.front();
            s->bulk.pop_front();
            r->reserve = std::min(bytes, s->bulk_budget);
            s->bulk_reserved += r->reserve;
            break;
          }
        }
        s->cv_bulk.wait(lk);
      }
      rpq::ctx_set_cancel(ctx, false);
    }
    r->t_start = Clock::now();
    rpq_set_option(ctx, "max_groups", G);
    int rc = RPQ_OK;
    uint64_t count = 0, dsum = 0, dxor = 0;
    rpq_result *res = nullptr;
    if (r->kind == RPQ_REQ_ALLPAIRS)
      rc = run_rpq(ctx, s->g, r->q, nullptr, 0, RPQ_COUNT_ONLY, &res);
    else
      rc = run_crpq(ctx, s->g, r->n_vars, r->var_label.empty() ? nullptr : r->var_label.data(), r->atoms.data(),
                    (uint32_t)r->atoms.size(), nullptr, 0, RPQ_COUNT_ONLY, &res);
    if (rc == RPQ_OK) {
      result_info(res, &count, nullptr, &dsum, &dxor);
      free_result(res);
    }
    // the workspace goes back to the device, so the next bulk request (on
    // either worker) can have the memory this one reserved
    rpq::ctx_release_workspace(ctx);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->bulk_reserved -= std::min(s->bulk_reserved, r->reserve);
      if (!r->cancelled) complete(s, r, rc, count, dsum, dxor);
    }
    s->cv_done.notify_all();
    s->cv_bulk.notify_all();
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
  const uint64_t budget = mem_budget_bytes ? mem_budget_bytes : (uint64_t)(free_b * 0.8);
  auto *s = new rpq_server;
  s->owner = ctx;
  s->g = g;
  // slots of the serving launch: max_batch, fewer if their visited and
  // result sets would take more than a quarter of the budget
  uint32_t slots = std::min<uint32_t>(max_batch, 1u << 16);
  while (slots > 64 && rpq::serve_engine_bytes(slots, SERVE_HASH_BITS) > budget / 4) slots /= 2;
  const uint64_t serve_b = rpq::serve_engine_bytes(slots, SERVE_HASH_BITS) + (256ull << 20);
  const uint64_t lane_b = (budget - std::min(budget, serve_b)) / 2;
  s->bulk_budget = budget - std::min(budget, serve_b + lane_b);
  s->lanes = 4096;
  s->slots = slots;
  int rc = RPQ_OK;
  for (auto &st : s->streams)
    if (rc == RPQ_OK && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) rc = RPQ_ERR_CUDA;
  if (rc == RPQ_OK) rc = rpq_create(&s->ctx_serve, dev, serve_b, s->streams[0]);
  if (rc == RPQ_OK) rc = rpq_create(&s->ctx_lane, dev, lane_b, s->streams[1]);
  for (int w = 0; w < BULK_WORKERS && rc == RPQ_OK; w++)
    rc = rpq_create(&s->ctx_bulk[w], dev, s->bulk_budget, s->streams[2 + w]);
  if (rc == RPQ_OK) {
    // the workers follow the owner's tunables and share the device
    for (rpq_ctx *c : {s->ctx_serve, s->ctx_lane, s->ctx_bulk[0], s->ctx_bulk[1]}) rpq::ctx_copy_tunables(c, ctx);
    rpq_set_option(s->ctx_serve, "grid_share", SHARE_SERVE);
    rpq_set_option(s->ctx_lane, "grid_share", SHARE_LANE);
    for (rpq_ctx *c : s->ctx_bulk) rpq_set_option(c, "grid_share", SHARE_BULK);
    rc = rpq::serve_engine_create(s->ctx_serve, g, slots, SERVE_HASH_BITS, SERVE_EVICT_AT, &s->eng);
  }
  if (rc != RPQ_OK) {
    std::string msg = s->ctx_serve ? rpq_last_error(s->ctx_serve) : "";
    for (rpq_ctx *c : {s->ctx_serve, s->ctx_lane, s->ctx_bulk[0], s->ctx_bulk[1]}) rpq_destroy(c);
    for (auto st : s->streams)
      if (st) cudaStreamDestroy(st);
    delete s;
    return rpq::ctx_error(ctx, rc, "server creation failed: " + msg);
  }
  s->t_single = std::thread(single_driver, s);
  s->t_lane = std::thread(lane_worker, s);
  for (int w = 0; w < BULK_WORKERS; w++) s->t_bulk[w] = std::thread(bulk_worker, s, w);
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
    if (raw->kind == RPQ_REQ_SINGLE) {
      if (rpq::query_host(raw->q).d.n_states == 0) {  // the empty language: no rows
        raw->t_start = raw->t_submit;
        complete(s, raw, RPQ_OK, 0, 0, 0);
      } else {
        s->singles.push_back(raw);
      }
    } else {
      s->bulk.push_back(raw);
    }
  }
  s->cv_work.notify_all();
  s->cv_bulk.notify_all();
  s->cv_done.notify_all();
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
  // a cancelled request still on the device is released when its reply arrives
  if (s->inflight.count(ticket))
    r->waited = true;
  else
    s->reqs.erase(it);
  return RPQ_OK;
}

int rpq_server_cancel(rpq_server *s) {
  if (!s) return RPQ_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (rpq_ctx *c : s->ctx_bulk) rpq::ctx_set_cancel(c, true);  // the bulk requests in service
    const auto now = Clock::now();
    auto cancel = [&](Req *r) {
      if (r->done) return;
      r->cancelled = true;
      r->status = RPQ_ERR_CANCELLED;
      if (r->t_start == Clock::time_point()) r->t_start = now;
      r->t_done = now;
      r->done = true;
    };
    for (auto *q : {&s->singles, &s->lane_q, &s->bulk}) {
      for (Req *r : *q) cancel(r);
      q->clear();
    }
    // singles already handed to the device: their replies are dropped
    for (auto &kv : s->inflight) cancel(kv.second);
  }
  s->cv_done.notify_all();
  s->cv_bulk.notify_all();
  return RPQ_OK;
}

int rpq_server_stats(rpq_server *s, uint64_t *batches, uint64_t *batched_requests) {
  if (!s) return RPQ_ERR_INVALID_ARG;
  uint64_t launches = 0, admitted = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    rpq::serve_engine_counters(s->eng, &launches, &admitted);
  }
  if (batches) *batches = launches;
  if (batched_requests) *batched_requests = admitted;
  return RPQ_OK;
}

int rpq_server_info(rpq_server *s, rpq_server_counters *out) {
  if (!s || !out) return RPQ_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  {
    std::lock_guard<std::mutex> lk(s->mu);
    rpq::serve_engine_counters(s->eng, &out->launches, &out->admitted);
  }
  out->lane_requests = s->lane_requests;
  out->lane_launches = s->lane_launches;
  out->graph = rpq::serve_engine_graphed(s->eng) ? 1u : 0u;
  out->slots = s->slots;
  return RPQ_OK;
}

void rpq_server_destroy(rpq_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  s->cv_lane.notify_all();
  s->cv_bulk.notify_all();
  if (s->t_single.joinable()) s->t_single.join();
  {
    std::lock_guard<std::mutex> lk(s->mu);
  }
  s->cv_lane.notify_all();
  if (s->t_lane.joinable()) s->t_lane.join();
  for (auto &t : s->t_bulk)
    if (t.joinable()) t.join();
  rpq::serve_engine_destroy(s->eng);
  for (rpq_ctx *c : {s->ctx_serve, s->ctx_lane, s->ctx_bulk[0], s->ctx_bulk[1]}) rpq_destroy(c);
  for (auto st : s->streams)
    if (st) cudaStreamDestroy(st);
  delete s;
}

}  // extern "C"
