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
};

struct BatchOut {
  uint64_t count = 0, dsum = 0, dxor = 0;
  rpq_stats stats{};
  std::vector<std::pair<u32 *, uint64_t>> chunks;  // row-major (query, vertex) rows, in order
  bool per_query = false;       // fill qstats: per query (rows, digest sum, digest xor) of its
  std::vector<uint64_t> qstats;  // (source, y) rows, as run_rpq would report them alone
  uint64_t evicted = 0;          // queries that left the batch for the multi-source engine
  std::vector<uint32_t> evicted_idx;
  uint64_t regroup_launches = 0; // multi-source evaluations (one per distinct automaton)
};

BatchTuning batch_default_tuning();
BatchTuning ctx_batch_tuning(rpq_ctx *ctx);  // the context's current tuning

// Evaluates queries[i] from sources[i] for i < nq; rows (i, y) sorted.
int batch_run(rpq_ctx *ctx, const rpq_graph *g, uint32_t nq, const rpq_query *const *queries,
              const uint32_t *sources, bool materialize, const BatchTuning &tun, BatchOut *out);

}  // namespace rpq
