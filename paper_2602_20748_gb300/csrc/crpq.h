// Interface between the host API and the CRPQ join module.
#pragma once

#include <string>
#include <vector>

#include "device_common.cuh"
#include "rpq_internal.h"

namespace rpq {

// Per-source result rows of one RPQ evaluation (device memory): lane i of
// the chunk is start vertex lanesrc[i] (0xFFFFFFFF = unused lane); its
// destinations, ascending, are dst[lane_off[i] .. lane_off[i + 1]).
struct RowChunk {
  u32 *lanesrc = nullptr;
  u64 *lane_off = nullptr;
  u32 *dst = nullptr;
  uint64_t rows = 0;
  uint32_t n_lanes = 0;
  // lanes whose rows are bitsets over the vertices (RowBitsReq): lane i's
  // bitset is bits + lane_slot[i] * bwords when lane_slot[i] != NO_SOURCE;
  // its destinations are listed in dst as well only when lists_kept
  u64 *bits = nullptr;
  u32 *lane_slot = nullptr;
  uint64_t bwords = 0;
  uint32_t n_bits = 0;
  bool lists_kept = true;
};

// Rows of at least min_len destinations come out as bitsets of the vertices
// (bwords 64-bit words each, bwords a multiple of 4), longest first while
// the chunk's bitsets take at most half of the budget left; keep_lists: such
// rows are listed in dst as well.
struct RowBitsReq {
  uint64_t min_len = 1;
  bool keep_lists = true;
};

int ctx_alloc(rpq_ctx *ctx, void **p, uint64_t bytes);
void ctx_free(rpq_ctx *ctx, void *p, uint64_t bytes);
cudaStream_t ctx_stream(rpq_ctx *ctx);
int ctx_error(rpq_ctx *ctx, int code, const std::string &msg);
int ctx_device(rpq_ctx *ctx);
int ctx_bfs_blocks(rpq_ctx *ctx, int nw);
int ctx_sm_share(rpq_ctx *ctx);  // SMs the context's persistent grids may use
float ctx_alpha(rpq_ctx *ctx);
double ctx_crpq_bitset_frac(rpq_ctx *ctx);  // rows of at least this fraction of the vertices get a bitset
uint64_t ctx_budget_left(rpq_ctx *ctx);     // budget bytes not allocated
bool ctx_trace(rpq_ctx *ctx);              // per-level trace printing (RPQ_TRACE=1)
// alpha, time limit, spill capacity and batched-engine tuning of `from`
void ctx_copy_tunables(rpq_ctx *to, const rpq_ctx *from);
// k helper contexts (created once, kept by ctx): own streams, ctx's budget
// / (k + 1) each and ctx->grid_share / k of the SMs, for evaluations that
// run side by side from k host threads.
int ctx_helpers(rpq_ctx *ctx, int k, std::vector<rpq_ctx *> *out);
// `count` pinned host buffers of `bytes` each, owned by the context and kept
// for reuse (one user at a time).
int ctx_pinned(rpq_ctx *ctx, int count, size_t bytes, void **out);
bool ctx_cancelled(rpq_ctx *ctx);          // a server asked the request in service to stop
void ctx_set_cancel(rpq_ctx *ctx, bool on);
uint64_t ctx_time_limit_ns(rpq_ctx *ctx);
// Device address of the static scratch array of run_rpq_static on the
// context's device (looked up by rpq_create).
void *ctx_static_scratch(rpq_ctx *ctx);
// Frees the context's traversal workspace and returns its pool's unused
// memory to the device (the next evaluation allocates afresh).
void ctx_release_workspace(rpq_ctx *ctx);
int static_scratch_prepare(void **addr, std::string *msg);
const DevGraph &graph_dev(const rpq_graph *g);
const HostQuery &query_host(const rpq_query *q);
int rpq_rows_for_sources(rpq_ctx *ctx, const rpq_graph *g, const rpq_query *q, std::vector<uint32_t> &srcs,
                         bool reverse, std::vector<RowChunk> *chunks, rpq_stats *stats, uint64_t *dsum = nullptr,
                         uint64_t *dxor = nullptr, const RowBitsReq *bits_req = nullptr);
void free_row_chunk(rpq_ctx *ctx, RowChunk &c);
// One automaton and at most 64 start vertices: a lane group of a
// multi-automaton launch.
struct MultiUnit {
  const rpq_query *q = nullptr;
  std::vector<uint32_t> srcs;
};
int rpq_lane_stats_multi(rpq_ctx *ctx, const rpq_graph *g, const std::vector<MultiUnit> &units,
                         std::vector<uint64_t> *lane_stats, rpq_stats *stats);
// One single-source task of a lane-mode launch: a query and its start vertex.
struct LaneTask {
  const rpq_query *q = nullptr;
  uint32_t source = 0;
};
// Count-only evaluation of single-source tasks with a different automaton per
// lane: tasks are packed up to max_lanes (<= 4,096) per launch, ordered by
// their automata's state counts; task i's own (rows, digest sum, digest xor)
// go to lane_stats[3 * i ..], counters are added to *stats.
// done_s (optional): per task, the host steady-clock time (s) at which its
// launch's summaries were read back.
int rpq_lane_stats_lanes(rpq_ctx *ctx, const rpq_graph *g, const std::vector<LaneTask> &tasks, uint32_t max_lanes,
                         std::vector<uint64_t> *lane_stats, rpq_stats *stats, std::vector<double> *done_s = nullptr);
double host_seconds();  // steady clock
int rpq_lane_stats_for_sources(rpq_ctx *ctx, const rpq_graph *g, const rpq_query *q,
                               const std::vector<uint32_t> &srcs, std::vector<uint64_t> *lane_stats,
                               rpq_stats *stats);
int make_tuple_result(rpq_ctx *ctx, uint32_t arity, u32 *tuples, uint64_t rows, uint64_t dsum, uint64_t dxor,
                      bool materialized, const rpq_stats &stats, rpq_result **out);

int crpq_eval(rpq_ctx *ctx, const rpq_graph *g, uint32_t n_vars, const int32_t *var_label, const crpq_atom *atoms,
              uint32_t n_atoms, const uint32_t *restrict0, uint32_t n_restrict0, uint32_t flags, rpq_result **out);

}  // namespace rpq
