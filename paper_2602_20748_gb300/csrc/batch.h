// Interface of the batched single-source engine (batch.cu).
#pragma once

#include <utility>
#include <vector>

#include "device_common.cuh"
#include "rpq_internal.h"

namespace rpq {

constexpr int RPQ_BATCH_SPLIT = 1;  // internal: the launch must be retried with fewer queries

// Tunables of the batched engine (chosen by rpq_autotune_batch).
struct BatchTuning {
  int threads;                  // block size of the persistent kernel
  uint32_t queries_per_launch;  // queries sharing one launch
  uint64_t list_cap;            // frontier list capacity (entries)
  uint64_t spill_cap;           // long-row chunks per level (<= SPILL_CAP)
  uint64_t evict_at;            // per-query mode: a query with more product vertices leaves the
                                // batch and is evaluated with the multi-source engine (0: never)
  bool multi;                   // evicted small automaton groups share multi-automaton launches
  uint32_t streams;             // helper contexts evaluating evicted queries side by side
  uint32_t lanes;               // per-query mode: evicted queries run in lane-mode launches of up to this
                                // many lanes, one automaton per lane (0: one bit-sliced launch per
                                // distinct automaton instead)
  bool direct;                  // per-query mode: every query goes straight to the lane-mode launches
  bool hash;                    // per-query mode: the shared launch keeps open-addressing visited sets
                                // (2 x evict_at slots per query) instead of dense bitmaps
};

struct BatchOut {
  uint64_t count = 0, dsum = 0, dxor = 0;
  rpq_stats stats{};
  std::vector<std::pair<u32 *, uint64_t>> chunks;  // row-major (query, vertex) rows, in order
  bool per_query = false;       // fill qstats: per query (rows, digest sum, digest xor) of its
  std::vector<uint64_t> qstats;  // (source, y) rows, as run_rpq would report them alone
  std::vector<double> qdone_ms;  // per query: ms from batch_run's start until its summary was known
  uint64_t evicted = 0;          // queries that left the batch for the multi-source engine
  std::vector<uint32_t> evicted_idx;
  uint64_t regroup_launches = 0; // multi-source evaluations (one per distinct automaton)
};

// ---- persistent serving launch ------------------------------------------
// Single-source requests enter a running launch: the host writes them into a
// ring in mapped host memory, and at every level boundary the launch takes
// as many as it has free slots (and reply room) for, seeds them and expands
// them with everything else in flight; a query whose frontier ran empty
// leaves its slot with its reply in a second ring, and one that grows past
// the eviction threshold (or fills its hash table) leaves it marked evicted
// (the host evaluates it elsewhere).  The launch ends when no slot is busy
// and nothing is waiting; the host launches it again when requests arrive.
struct ServeReq {               // one request (written by the host)
  unsigned long long ticket;
  unsigned int source;
  unsigned int pad;
  QueryDesc qd;
};
struct ServeDone {              // one reply (written by the device)
  unsigned long long ticket;
  unsigned long long count, dsum, dxor;  // the (source, y) rows: count and digest
  unsigned long long product_vertices, product_edges;
  unsigned int evicted;         // 1: the query left the launch; its result is not here
  unsigned int pad;
};
struct ServeShared {            // mapped host memory shared by host and device
  volatile unsigned long long req_tail;   // host: requests written
  volatile unsigned long long req_head;   // device: requests taken
  volatile unsigned long long done_tail;  // device: replies written
  volatile unsigned long long done_head;  // host: replies consumed
  volatile unsigned int stop;             // host: admit nothing more
  unsigned int pad;
};
struct ServeEngine;
struct ServeReply {
  uint64_t ticket, count, dsum, dxor, product_vertices, product_edges;
  bool evicted;
};
// slots: queries in flight at once; hash_bits: log2 of each slot's visited
// (and result) table; evict_at: product vertices after which a query leaves.
int serve_engine_create(rpq_ctx *ctx, const rpq_graph *g, uint32_t slots, uint32_t hash_bits, uint64_t evict_at,
                        ServeEngine **out);
void serve_engine_destroy(ServeEngine *e);
// Device bytes the engine holds (for admission accounting).
uint64_t serve_engine_bytes(uint32_t slots, uint32_t hash_bits);
// Queues a request in the ring; false when the ring is full.
bool serve_engine_push(ServeEngine *e, uint64_t ticket, const QueryDesc &qd, uint32_t source);
// Requests written but not yet taken by the device.
uint64_t serve_engine_waiting(ServeEngine *e);
// Takes the replies written so far.
void serve_engine_poll(ServeEngine *e, std::vector<ServeReply> *out);
// Launches the serving kernel if it is not running and requests are waiting.
// Returns RPQ_OK, or an error code once a launch has failed (its requests are
// then lost: *lost gets their tickets, and the engine is reset).
int serve_engine_kick(ServeEngine *e, std::vector<uint64_t> *lost);
bool serve_engine_running(ServeEngine *e);
// Whether relaunches go through a captured CUDA graph.
bool serve_engine_graphed(ServeEngine *e);
// Launches so far and levels run.
void serve_engine_counters(ServeEngine *e, uint64_t *launches, uint64_t *admitted);

BatchTuning batch_default_tuning();
BatchTuning ctx_batch_tuning(rpq_ctx *ctx);  // the context's current tuning

// Evaluates queries[i] from sources[i] for i < nq; rows (i, y) sorted.
int batch_run(rpq_ctx *ctx, const rpq_graph *g, uint32_t nq, const rpq_query *const *queries,
              const uint32_t *sources, bool materialize, const BatchTuning &tun, BatchOut *out);

}  // namespace rpq
