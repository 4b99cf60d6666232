// Host side of the C ABI declared in include/rpq.h: contexts, device memory
// budget, graph loading, query compilation, batched evaluation driving the
// traversal and emission kernels, results and fetch.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <chrono>

#include "batch.h"
#include "crpq.h"
#include "device_common.cuh"
#include "rpq_internal.h"

using namespace rpq;

namespace {

thread_local std::string g_create_error;

constexpr int BFS_THREADS_HOST = 256;
constexpr size_t SOURCE_FILTER_MIN = 4096;  // source lists at least this long drop edgeless start vertices

struct Workspace {
  uint64_t vis_words = 0;   // capacity of vis / fr0 / fr1 in u64 words
  uint64_t list_cap = 0;    // capacity of list0 / list1 in entries
  uint64_t claim_cap = 0;   // capacity of claim in u32
  uint32_t lane_cap = 0;    // lanesrc / empty-mask staging capacity (lanes)
  u64 *vis = nullptr, *fr0 = nullptr, *fr1 = nullptr, *list0 = nullptr, *list1 = nullptr;
  u32 *claim = nullptr;
  u32 *lanesrc = nullptr;
  u64 *empty = nullptr;
  u64 *spill = nullptr;  // SPILL_CAP chunk records of 6 words
  u32 *fbits = nullptr;  // two frontier bitmaps of fbits_words() words each
  uint64_t fbits_words() const { return (list_cap + 31) / 32; }  // list_cap >= Q * n
};

}  // namespace

struct rpq_ctx {
  int device = -1;
  cudaStream_t stream = nullptr;
  cudaMemPool_t pool = nullptr;  // the context's own pool: freed blocks stay reserved for reuse
  uint64_t budget = 0;
  uint64_t used = 0;
  std::string err;
  Workspace ws;
  BfsCtl *ctl = nullptr;
  u64 *small = nullptr;  // [0..1] digest, [2] total, [3..7] spare
  uint32_t stamp = 0;
  int sms = 0;
  int bpsm[2] = {0, 0};  // resident traversal blocks per SM for NW = 1, 4
  int bpsm_multi = 0;    // the same for the per-group-automata kernel (set on first use)
  int bpsm_lane[2] = {0, 0};  // and for the per-lane-automata kernel, NW = 1, 4 (set on first use)
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  float alpha = 16.0f;
  float lane_alpha = 2.0f;  // the same trade-off for lane-mode launches
  unsigned pull_dynamic = 1;  // bottom-up vertex chunks from a cursor
  unsigned lane_by_source = 1;  // lane-mode light rows gathered per (label, source state)
  double crpq_bitset_frac = 1.0 / 64;  // CRPQ rows of at least this fraction of the vertices get a bitset
  uint64_t time_limit_ns = 20ull * 1000 * 1000 * 1000;
  uint32_t max_groups = 16;
  bool trace = false;    // print per-level timings of each traversal (RPQ_TRACE=1)
  uint64_t spill_cap = SPILL_CAP;  // long-row chunks per level (RPQ_SPILL_CAP lowers it)
  double grid_share = 1.0;         // fraction of the SMs persistent grids use
  rpq::BatchTuning batch = rpq::batch_default_tuning();  // run_rpq_batch tunables
  std::atomic<int> cancel{0};  // set by a server to stop the request in service
  std::vector<void *> pinned;  // pinned host slots lent to streams (kept for reuse)
  unsigned char *rb_host = nullptr;  // mapped pinned read-back buffer (RB_CAP bytes)
  void *rb_dev = nullptr;            // its device address
  std::vector<rpq_ctx *> helpers;  // contexts for concurrent sub-evaluations (own streams)
  std::vector<cudaStream_t> helper_streams;
  size_t pinned_bytes = 0;
  int live = 0;          // graphs and results not yet freed
  bool closing = false;  // rpq_destroy was called while handles were live
  void *static_scratch = nullptr;  // device address of run_rpq_static's array
};

struct rpq_graph {
  rpq_ctx *ctx = nullptr;
  DevGraph g;
  uint64_t bytes = 0;
};

struct rpq_query {
  HostQuery hq;
};

namespace {

struct Chunk {
  u32 *lanesrc = nullptr;
  u64 *lane_off = nullptr;
  u32 *dst = nullptr;
  uint64_t rows = 0;
  uint32_t n_lanes = 0;
  uint64_t bytes = 0;
  u64 *bits = nullptr;  // bitset rows (see RowChunk)
  u32 *lane_slot = nullptr;
  uint64_t bwords = 0;
  uint32_t n_bits = 0;
  bool lists_kept = true;
};

}  // namespace

struct rpq_result {
  rpq_ctx *ctx = nullptr;
  uint32_t arity = 2;
  uint64_t count = 0;
  uint64_t dsum = 0, dxor = 0;
  bool materialized = false;
  std::vector<Chunk> chunks;
  u32 *tuples = nullptr;  // CRPQ rows, arity values each
  uint64_t tuple_bytes = 0;
  rpq_stats stats;
  std::vector<uint64_t> qstats;  // run_rpq_batch with RPQ_PER_QUERY: 3 values per query
  std::vector<double> qdone_ms;  // and when each query's summary was known (ms from the call's start)
};

namespace {

int set_err(rpq_ctx *c, int code, const std::string &msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_err(rpq_ctx *c, cudaError_t e, const char *what) {
  return set_err(c, RPQ_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(expr)                                          \
  do {                                                    \
    cudaError_t _e = (expr);                              \
    if (_e != cudaSuccess) return cuda_err(ctx, _e, #expr); \
  } while (0)

int dev_alloc(rpq_ctx *ctx, void **p, uint64_t bytes) {
  if (bytes == 0) bytes = 16;
  if (ctx->used + bytes > ctx->budget)
    return set_err(ctx, RPQ_ERR_OUT_OF_BUDGET,
                   "device memory budget exceeded (" + std::to_string(ctx->used + bytes) + " > " +
                       std::to_string(ctx->budget) + " bytes)");
  cudaError_t e = ctx->pool ? cudaMallocFromPoolAsync(p, bytes, ctx->pool, ctx->stream)
                            : cudaMallocAsync(p, bytes, ctx->stream);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_err(ctx, e, "stream-ordered allocation");
  }
  ctx->used += bytes;
  return RPQ_OK;
}

void dev_free(rpq_ctx *ctx, void *p, uint64_t bytes) {
  if (!p) return;
  if (bytes == 0) bytes = 16;
  cudaFreeAsync(p, ctx->stream);
  ctx->used -= std::min(ctx->used, bytes);
}

template <typename T>
int dalloc(rpq_ctx *ctx, T **p, uint64_t count) {
  return dev_alloc(ctx, (void **)p, count * sizeof(T));
}

template <typename T>
void dfree(rpq_ctx *ctx, T *&p, uint64_t count) {
  dev_free(ctx, (void *)p, count * sizeof(T));
  p = nullptr;
}

// Small device -> host reads (the traversal's control block, totals, source
// flags) go through a kernel into a mapped pinned buffer instead of the copy
// engines: a stream's bulk row copies queued there would otherwise hold every
// such read back until they drain.
constexpr size_t RB_CAP = 1u << 20;

__global__ void rb_copy_kernel(unsigned char *__restrict__ dst, const unsigned char *__restrict__ src, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

// Queues the copy of `bytes` (off + bytes <= RB_CAP) from device memory src to
// read-back offset off; the bytes are at ctx->rb_host + off once the stream is
// synchronized.
cudaError_t rb_queue(rpq_ctx *ctx, size_t off, const void *src, size_t bytes) {
  if (!ctx->rb_host) {
    void *h = nullptr;
    cudaError_t e = cudaHostAlloc(&h, RB_CAP, cudaHostAllocMapped);
    if (e != cudaSuccess) return e;
    if ((e = cudaHostGetDevicePointer(&ctx->rb_dev, h, 0)) != cudaSuccess) {
      cudaFreeHost(h);
      return e;
    }
    ctx->rb_host = static_cast<unsigned char *>(h);
  }
  if (bytes == 0) return cudaSuccess;
  if (off + bytes > RB_CAP) return cudaErrorInvalidValue;
  const unsigned blocks = (unsigned)std::min<size_t>((bytes + 255) / 256, 1024);
  rb_copy_kernel<<<blocks, 256, 0, ctx->stream>>>(static_cast<unsigned char *>(ctx->rb_dev) + off,
                                                  static_cast<const unsigned char *>(src), bytes);
  return cudaGetLastError();
}

constexpr size_t RB_SMALL = (sizeof(BfsCtl) + 15) & ~(size_t)15;  // read-back offset after the control block

bool usable(rpq_ctx *ctx) {
  if (!ctx) return false;
  if (ctx->device < 0) {
    set_err(ctx, RPQ_ERR_NO_DEVICE, "host-only context has no GPU");
    return false;
  }
  cudaSetDevice(ctx->device);
  return true;
}

void free_workspace(rpq_ctx *ctx) {
  Workspace &w = ctx->ws;
  dfree(ctx, w.vis, w.vis_words);
  dfree(ctx, w.fr0, w.vis_words);
  dfree(ctx, w.fr1, w.vis_words);
  dfree(ctx, w.list0, w.list_cap);
  dfree(ctx, w.list1, w.list_cap);
  dfree(ctx, w.claim, w.claim_cap);
  dfree(ctx, w.lanesrc, w.lane_cap);
  dfree(ctx, w.empty, w.lane_cap / 64 + 1);
  dfree(ctx, w.spill, SPILL_CAP * 6);
  dfree(ctx, w.fbits, 2 * w.fbits_words());
  w = Workspace();
}

uint64_t workspace_bytes(uint64_t words, uint64_t lists, uint64_t claims, uint32_t lanes) {
  return words * 8 * 3 + lists * 8 * 2 + (lists + 31) / 32 * 8 + claims * 4 + (uint64_t)lanes * 4 +
         (uint64_t)lanes / 64 * 8;
}

// Makes sure the traversal workspace holds at least the given capacities.
// Frontier arrays must be zero on entry to a search; they are zeroed when
// allocated and the search leaves them zero.
int ensure_workspace(rpq_ctx *ctx, uint64_t words, uint64_t lists, uint64_t claims, uint32_t lanes) {
  Workspace &w = ctx->ws;
  if (w.vis_words >= words && w.list_cap >= lists && w.claim_cap >= claims && w.lane_cap >= lanes) return RPQ_OK;
  words = std::max(words, w.vis_words);
  lists = std::max(lists, w.list_cap);
  claims = std::max(claims, w.claim_cap);
  lanes = std::max(lanes, w.lane_cap);
  free_workspace(ctx);
  // capacities first, so that a failed allocation releases what it got
  w.vis_words = words;
  w.list_cap = lists;
  w.claim_cap = claims ? claims : 1;
  w.lane_cap = lanes;
  int rc;
  if ((rc = dalloc(ctx, &w.vis, words)) || (rc = dalloc(ctx, &w.fr0, words)) || (rc = dalloc(ctx, &w.fr1, words)) ||
      (rc = dalloc(ctx, &w.list0, lists)) || (rc = dalloc(ctx, &w.list1, lists)) ||
      (rc = dalloc(ctx, &w.claim, claims ? claims : 1)) || (rc = dalloc(ctx, &w.lanesrc, lanes)) ||
      (rc = dalloc(ctx, &w.empty, lanes / 64 + 1)) || (rc = dalloc(ctx, &w.spill, SPILL_CAP * 6)) ||
      (rc = dalloc(ctx, &w.fbits, 2 * ((lists + 31) / 32)))) {
    free_workspace(ctx);
    return rc;
  }
  CK(cudaMemsetAsync(w.fbits, 0, 2 * w.fbits_words() * 4, ctx->stream));
  CK(cudaMemsetAsync(w.fr0, 0, words * 8, ctx->stream));
  CK(cudaMemsetAsync(w.fr1, 0, words * 8, ctx->stream));
  CK(cudaMemsetAsync(w.claim, 0, w.claim_cap * 4, ctx->stream));
  ctx->stamp = 0;
  return RPQ_OK;
}

// A traversal launch stopped early: clear what it may have left set (the
// frontier words and bitmaps must be zero for the next search) and map the
// device error word to an error code.
int traversal_error(rpq_ctx *ctx, unsigned err) {
  Workspace &w = ctx->ws;
  cudaMemsetAsync(w.fr0, 0, w.vis_words * 8, ctx->stream);
  cudaMemsetAsync(w.fr1, 0, w.vis_words * 8, ctx->stream);
  cudaMemsetAsync(w.fbits, 0, 2 * w.fbits_words() * 4, ctx->stream);
  if (err == ERR_LIST_OVERFLOW) return set_err(ctx, RPQ_ERR_CUDA, "internal: traversal entry list overflow");
  return set_err(ctx, RPQ_ERR_TIMEOUT, "traversal grid barrier wait ran out of time");
}

void free_chunk(rpq_ctx *ctx, Chunk &c) {
  dfree(ctx, c.lanesrc, c.n_lanes);
  dfree(ctx, c.lane_off, (uint64_t)c.n_lanes + 1);
  dfree(ctx, c.dst, c.rows);
  if (c.bits) {
    dfree(ctx, c.bits, (uint64_t)c.n_bits * c.bwords);
    dfree(ctx, c.lane_slot, c.n_lanes);
  }
}

// Picks the lanes of a chunk whose rows become bitsets (bits_req): reads the
// lanes' row counts from the scanned offsets, keeps the rows of at least
// min_len destinations, longest first, while the bitsets take at most half of
// the budget left, and allocates them into c.  Returns the lanes' slots on
// the host (NO_SOURCE: listed only).
int pick_bit_lanes(rpq_ctx *ctx, const RowBitsReq &req, const u64 *off, uint32_t segs, uint32_t n, Chunk &c) {
  std::vector<u64> lane_off(c.n_lanes + 1);
  u64 *d_lane_off = nullptr;
  int rc;
  if ((rc = dalloc(ctx, &d_lane_off, (uint64_t)c.n_lanes + 1))) return rc;
  cudaError_t e = launch_gather_lane_off(off, segs, c.n_lanes, ctx->small + 2, d_lane_off, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(lane_off.data(), d_lane_off, lane_off.size() * 8, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  dfree(ctx, d_lane_off, (uint64_t)c.n_lanes + 1);
  if (e != cudaSuccess) return cuda_err(ctx, e, "row lengths");
  std::vector<uint32_t> sel;
  for (uint32_t i = 0; i < c.n_lanes; i++)
    if (lane_off[i + 1] - lane_off[i] >= std::max<uint64_t>(req.min_len, 1)) sel.push_back(i);
  if (sel.empty()) return RPQ_OK;
  std::stable_sort(sel.begin(), sel.end(), [&](uint32_t a, uint32_t b) {
    return lane_off[a + 1] - lane_off[a] > lane_off[b + 1] - lane_off[b];
  });
  const uint64_t bwords = ((uint64_t)n + 255) / 256 * 4;
  const uint64_t left = ctx->used < ctx->budget ? ctx->budget - ctx->used : 0;
  const uint64_t cap = left / 2 / (bwords * 8);
  if (sel.size() > cap) sel.resize(cap);
  if (sel.empty()) return RPQ_OK;
  std::vector<uint32_t> slot(c.n_lanes, NO_SOURCE);
  for (size_t k = 0; k < sel.size(); k++) slot[sel[k]] = (uint32_t)k;
  if ((rc = dalloc(ctx, &c.bits, sel.size() * bwords))) return rc;
  if ((rc = dalloc(ctx, &c.lane_slot, c.n_lanes))) {
    dfree(ctx, c.bits, sel.size() * bwords);
    c.bits = nullptr;
    return rc;
  }
  c.n_bits = (uint32_t)sel.size();
  c.bwords = bwords;
  c.lists_kept = req.keep_lists;
  e = cudaMemcpyAsync(c.lane_slot, slot.data(), (uint64_t)c.n_lanes * 4, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);  // slot is a host temporary
  if (e != cudaSuccess) return cuda_err(ctx, e, "bitset slots");
  return RPQ_OK;
}

// Evaluates one RPQ from the sorted, distinct start vertices `srcs`.
// With lane_stats (count-only), (rows, digest sum, digest xor) of every
// source's own rows are stored at lane_stats[3 * i ..] for srcs[i].
int eval_rpq(rpq_ctx *ctx, const rpq_graph *gr, const rpq_query *qr, const std::vector<uint32_t> &srcs_in,
             uint32_t flags, rpq_result *res, std::vector<uint64_t> *lane_stats = nullptr,
             const RowBitsReq *bits_req = nullptr) {
  const DevGraph &g = gr->g;
  const bool reverse = (flags & RPQ_REVERSE) != 0;
  if (reverse && !qr->hq.has_rev)
    return set_err(ctx, RPQ_ERR_TOO_COMPLEX, "the reversed language needs more than RPQ_MAX_STATES states");
  const QueryDesc &qd = reverse ? qr->hq.rev : qr->hq.d;
  const uint32_t Q = qd.n_states;
  const bool materialize = (flags & RPQ_MATERIALIZE) != 0;
  if (lane_stats) lane_stats->assign(3 * srcs_in.size(), 0);
  if (Q == 0 || srcs_in.empty()) {
    res->stats.lane_words = srcs_in.size() <= 64 ? 1 : 4;
    return RPQ_OK;
  }
  // A start vertex with no edge on a label leaving the start state reaches
  // only (s, q0): its one possible row is (s, s), when q0 accepts.  Large
  // source lists drop such vertices before the traversal (their rows are
  // added here), unless rows are kept and q0 accepts (the (s, s) rows would
  // have to be interleaved with the others).
  std::vector<uint32_t> kept;
  const bool q0_final = (qd.final_mask & 1u) != 0;
  const bool filter = !lane_stats && srcs_in.size() >= SOURCE_FILTER_MIN && !(q0_final && materialize);
  if (filter) {
    unsigned long long lmask = 0;
    for (uint32_t t = qd.out_begin[0]; t < qd.out_begin[1]; t++)
      if (qd.out_label[t] < 64) lmask |= 1ull << qd.out_label[t];
    u32 *dsrc = nullptr;
    unsigned char *dflag = nullptr;
    int rc2;
    if ((rc2 = dalloc(ctx, &dsrc, srcs_in.size()))) return rc2;
    if ((rc2 = dalloc(ctx, &dflag, srcs_in.size()))) {
      dfree(ctx, dsrc, srcs_in.size());
      return rc2;
    }
    std::vector<unsigned char> flag(srcs_in.size());
    cudaError_t e = cudaMemcpyAsync(dsrc, srcs_in.data(), srcs_in.size() * 4, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
      e = launch_source_filter(reverse ? g.in_off : g.out_off, g.n, g.L, lmask, dsrc, srcs_in.size(), dflag,
                               ctx->stream);
    const bool rb = srcs_in.size() <= RB_CAP;
    if (e == cudaSuccess)
      e = rb ? rb_queue(ctx, 0, dflag, srcs_in.size())
             : cudaMemcpyAsync(flag.data(), dflag, srcs_in.size(), cudaMemcpyDeviceToHost, ctx->stream);
    dfree(ctx, dsrc, srcs_in.size());
    dfree(ctx, dflag, srcs_in.size());
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "source filter");
    if (rb) std::memcpy(flag.data(), ctx->rb_host, srcs_in.size());
    res->stats.launches += rb ? 2 : 1;
    kept.reserve(srcs_in.size());
    uint64_t skipped = 0;
    for (size_t i = 0; i < srcs_in.size(); i++) {
      if (flag[i]) {
        kept.push_back(srcs_in[i]);
        continue;
      }
      skipped++;
      if (q0_final) {
        const uint64_t h = splitmix64(((uint64_t)srcs_in[i] << 32) | srcs_in[i]);
        res->dsum += h;
        res->dxor ^= h;
      }
    }
    res->stats.product_vertices += skipped;
    if (q0_final) res->count += skipped;
  }
  const std::vector<uint32_t> &srcs = filter ? kept : srcs_in;
  res->stats.lane_words = srcs.size() <= 64 ? 1 : 4;
  if (srcs.empty()) return RPQ_OK;
  const int nw = srcs.size() <= 64 ? 1 : 4;
  const uint32_t K = 64u * nw;
  const uint32_t n = g.n;
  const uint64_t groups_total = (srcs.size() + K - 1) / K;

  const int force = (flags & RPQ_FORCE_PUSH) ? 1 : (flags & RPQ_FORCE_PULL) ? 2 : 0;
  const int blocks = ctx_bfs_blocks(ctx, nw);
  if (blocks <= 0) return set_err(ctx, RPQ_ERR_CUDA, "traversal kernel cannot be made resident");
  // list slots a level can leave unused: every warp may end each of the two
  // appending phases of a level with part of a reserved segment
  const uint64_t slack = 2ull * blocks * (BFS_THREADS_HOST / 32) * APPEND_SEG;

  // lane groups per launch: bounded by max_groups and by the budget
  uint32_t G = (uint32_t)std::min<uint64_t>(groups_total, ctx->max_groups);
  for (;;) {
    uint64_t words = (uint64_t)G * Q * n * nw;
    uint64_t need = workspace_bytes(words, (uint64_t)G * Q * n + slack, nw > 1 ? (uint64_t)G * Q * n : 0, G * K);
    uint64_t have = ctx->budget - ctx->used +
                    workspace_bytes(ctx->ws.vis_words, ctx->ws.list_cap, ctx->ws.claim_cap, ctx->ws.lane_cap);
    if (need + (64ull << 20) <= have || G == 1) break;
    G--;
  }
  {
    uint64_t words = (uint64_t)G * Q * n * nw;
    int rc = ensure_workspace(ctx, words, (uint64_t)G * Q * n + slack, nw > 1 ? (uint64_t)G * Q * n : 0, G * K);
    if (rc) return rc;
  }
  Workspace &w = ctx->ws;
  const uint32_t segs = (n + EMIT_SEG - 1) / EMIT_SEG;

  std::vector<uint32_t> lanes;
  std::vector<uint64_t> empty;
  for (uint64_t g0 = 0; g0 < groups_total; g0 += G) {
    if (ctx->cancel.load(std::memory_order_relaxed)) return set_err(ctx, RPQ_ERR_CANCELLED, "cancelled");
    const uint32_t Gb = (uint32_t)std::min<uint64_t>(G, groups_total - g0);
    const uint32_t n_lanes = Gb * K;
    lanes.assign(n_lanes, NO_SOURCE);
    empty.assign((size_t)Gb * nw, 0);
    for (uint32_t i = 0; i < n_lanes; i++) {
      uint64_t si = g0 * K + i;
      if (si < srcs.size()) lanes[i] = srcs[si];
      if (lanes[i] == NO_SOURCE) empty[(i / K) * nw + (i % K) / 64] |= 1ull << (i % 64);
    }
    CK(cudaMemcpyAsync(w.lanesrc, lanes.data(), n_lanes * 4, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(w.empty, empty.data(), empty.size() * 8, cudaMemcpyHostToDevice, ctx->stream));

    BfsParams p;
    std::memset(&p, 0, sizeof(p));
    // the reverse traversal is the forward one on the transposed graph
    p.out_off = reverse ? g.in_off : g.out_off;
    p.out_col = reverse ? g.in_col : g.out_col;
    p.in_off = reverse ? g.out_off : g.in_off;
    p.in_col = reverse ? g.out_col : g.in_col;
    // bottom-up levels read the in-direction of the traversal
    p.hchunk = reverse ? g.hchunk_out : g.hchunk_in;
    {
      const std::vector<uint32_t> &ho = reverse ? g.hchunk_out_off : g.hchunk_in_off;
      for (uint32_t l = 0; l <= g.L && l < ho.size(); l++) p.hchunk_off[l] = ho[l];
      for (uint32_t l = 0; l < g.L; l++) p.label_edges[l] = g.label_edges[l];
    }
    p.n = n;
    p.L = g.L;
    p.G = Gb;
    p.Q = Q;
    p.lanesrc = w.lanesrc;
    p.vis = w.vis;
    p.fr0 = w.fr0;
    p.fr1 = w.fr1;
    p.claim = w.claim;
    p.fbits = w.fbits;
    p.fbits_words = w.fbits_words();
    p.append_seg = APPEND_SEG;
    p.list_cap = w.list_cap;
    p.spill = w.spill;
    p.spill_cap = ctx->spill_cap;
    p.list0 = w.list0;
    p.list1 = w.list1;
    p.ctl = ctx->ctl;
    p.stamp_base = ctx->stamp;
    p.nblocks = (unsigned)blocks;
    p.force = force;
    p.alpha = ctx->alpha;
    p.pull_dynamic = ctx->pull_dynamic;
    p.lane_by_source = ctx->lane_by_source;
    p.time_limit_ns = ctx->time_limit_ns;
    p.q = qd;

    CK(launch_vis_init(nw, p, w.empty, ctx->stream));
    CK(cudaMemsetAsync(ctx->ctl, 0, sizeof(BfsCtl), ctx->stream));
    CK(cudaEventRecord(ctx->ev[0], ctx->stream));
    CK(launch_msbfs(nw, p, blocks, BFS_THREADS_HOST, ctx->stream));
    CK(cudaEventRecord(ctx->ev[1], ctx->stream));
    res->stats.launches += 3;
    res->stats.bfs_launches += 1;

    if (lane_stats && !materialize) {
      // per-lane summaries instead of the count pass
      u64 *ls = nullptr;
      int rc2 = dalloc(ctx, &ls, 3ull * n_lanes);
      if (rc2) return rc2;
      EmitParams ep{};
      std::memset(&ep, 0, sizeof(ep));
      ep.vis = w.vis;
      ep.n = n;
      ep.G = Gb;
      ep.Q = Q;
      ep.final_mask = qd.final_mask;
      ep.lanesrc = w.lanesrc;
      ep.segs = segs;
      CK(cudaMemsetAsync(ls, 0, 24ull * n_lanes, ctx->stream));
      CK(cudaEventRecord(ctx->ev[2], ctx->stream));
      CK(launch_emit_lane_stats(nw, ep, ls, ctx->stream));
      CK(cudaEventRecord(ctx->ev[3], ctx->stream));
      res->stats.launches += 1;
      std::vector<uint64_t> hls(3ull * n_lanes);
      BfsCtl hctl;
      CK(cudaMemcpyAsync(&hctl, ctx->ctl, sizeof(BfsCtl), cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaMemcpyAsync(hls.data(), ls, 24ull * n_lanes, cudaMemcpyDeviceToHost, ctx->stream));
      dfree(ctx, ls, 3ull * n_lanes);
      CK(cudaStreamSynchronize(ctx->stream));
      if (hctl.err) return traversal_error(ctx, hctl.err);
      for (uint32_t i = 0; i < n_lanes; i++) {
        const uint64_t si = g0 * K + i;
        if (si >= srcs.size()) break;
        (*lane_stats)[3 * si] = hls[3 * i];
        (*lane_stats)[3 * si + 1] = hls[3 * i + 1];
        (*lane_stats)[3 * si + 2] = hls[3 * i + 2];
        res->count += hls[3 * i];
        res->dsum += hls[3 * i + 1];
        res->dxor ^= hls[3 * i + 2];
      }
      rpq_stats &s = res->stats;
      s.product_edges += hctl.stats[ST_W];
      s.product_vertices += hctl.stats[ST_N];
      s.levels += hctl.levels;
      s.push_levels += hctl.stats[ST_PUSH_LEVELS];
      s.pull_levels += hctl.stats[ST_PULL_LEVELS];
      s.group_edges += hctl.stats[ST_GROUP_EDGES];
      s.group_rows += hctl.stats[ST_GROUP_ROWS];
      s.group_vertices += hctl.stats[ST_GROUP_VERTICES];
      s.pull_edges += hctl.stats[ST_PULL_EDGES];
      s.pull_vertices += hctl.stats[ST_PULL_VERTICES];
      s.alg_bytes += hctl.stats[ST_ALG_BYTES];
      s.group_product_edges += hctl.stats[ST_GROUP_W];
      s.group_label_rows += hctl.stats[ST_GROUP_X];
      s.lane_groups += Gb;
      ctx->stamp += (uint32_t)hctl.levels + 3;
      float ms_bfs = 0, ms_emit = 0;
      cudaEventElapsedTime(&ms_bfs, ctx->ev[0], ctx->ev[1]);
      cudaEventElapsedTime(&ms_emit, ctx->ev[2], ctx->ev[3]);
      s.bfs_ms += ms_bfs;
      s.emit_ms += ms_emit;
      continue;
    }

    // emission pass 1: counts and digest
    u32 *cnt = nullptr;
    u64 *off = nullptr, *tmp = nullptr;
    const uint64_t ncnt = (uint64_t)n_lanes * segs;
    const uint64_t tmpw = scan_tmp_words(ncnt);
    int rc;
    if ((rc = dalloc(ctx, &cnt, ncnt)) || (rc = dalloc(ctx, &off, ncnt)) || (rc = dalloc(ctx, &tmp, tmpw))) {
      dfree(ctx, cnt, ncnt);
      dfree(ctx, off, ncnt);
      dfree(ctx, tmp, tmpw);
      return rc;
    }
    EmitParams ep{};
    ep.vis = w.vis;
    ep.n = n;
    ep.G = Gb;
    ep.Q = Q;
    ep.final_mask = qd.final_mask;
    ep.lanesrc = w.lanesrc;
    ep.segs = segs;
    ep.cnt = cnt;
    ep.off = off;
    ep.dst = nullptr;
    ep.digest = ctx->small;
    CK(cudaMemsetAsync(ctx->small, 0, 3 * 8, ctx->stream));
    CK(cudaEventRecord(ctx->ev[2], ctx->stream));
    CK(launch_emit(nw, false, !materialize, ep, ctx->stream));
    CK(exclusive_scan_u32_to_u64(cnt, off, ncnt, ctx->small + 2, tmp, ctx->stream));
    res->stats.launches += 2;
    BfsCtl hctl;
    u64 hsmall[3];
    CK(rb_queue(ctx, 0, ctx->ctl, sizeof(BfsCtl)));
    CK(rb_queue(ctx, RB_SMALL, ctx->small, 3 * 8));
    res->stats.launches += 2;
    CK(cudaStreamSynchronize(ctx->stream));
    std::memcpy(&hctl, ctx->rb_host, sizeof(BfsCtl));
    std::memcpy(hsmall, ctx->rb_host + RB_SMALL, 3 * 8);
    if (hctl.err) {
      dfree(ctx, cnt, ncnt);
      dfree(ctx, off, ncnt);
      dfree(ctx, tmp, tmpw);
      return traversal_error(ctx, hctl.err);
    }
    const uint64_t total = hsmall[2];
    res->count += total;
    if (!materialize) {  // the count pass folded the digest
      res->dsum += hsmall[0];
      res->dxor ^= hsmall[1];
    }
    u64 hdig[2] = {0, 0};
    rpq_stats &s = res->stats;
    s.product_edges += hctl.stats[ST_W];
    s.product_vertices += hctl.stats[ST_N];
    s.levels += hctl.levels;
    s.push_levels += hctl.stats[ST_PUSH_LEVELS];
    s.pull_levels += hctl.stats[ST_PULL_LEVELS];
    s.group_edges += hctl.stats[ST_GROUP_EDGES];
    s.group_rows += hctl.stats[ST_GROUP_ROWS];
    s.group_vertices += hctl.stats[ST_GROUP_VERTICES];
    s.pull_edges += hctl.stats[ST_PULL_EDGES];
    s.pull_vertices += hctl.stats[ST_PULL_VERTICES];
    s.alg_bytes += hctl.stats[ST_ALG_BYTES];
      s.group_product_edges += hctl.stats[ST_GROUP_W];
      s.group_label_rows += hctl.stats[ST_GROUP_X];
    s.lane_groups += Gb;
    if (ctx->trace) {
      uint32_t nl = (uint32_t)std::min<uint64_t>(hctl.levels, TRACE_LEVELS);
      std::fprintf(stderr, "[rpq trace] G=%u Q=%u levels=%llu W=%llu\n", Gb, Q, (unsigned long long)hctl.levels,
                   (unsigned long long)hctl.stats[ST_W]);
      for (uint32_t l = 0; l < nl; l++)
        std::fprintf(stderr, "[rpq trace]   level %2u %s n=%10llu mf=%12llu %9.3f ms (commit %7.3f ms)\n", l,
                     hctl.trace_mode[l] == 1 ? "push" : "pull", (unsigned long long)hctl.trace_n[l],
                     (unsigned long long)hctl.trace_mf[l], (hctl.trace_t[l + 1] - hctl.trace_t[l]) * 1e-6,
                     hctl.trace_c[l] ? (hctl.trace_t[l + 1] - hctl.trace_c[l]) * 1e-6 : 0.0);
    }
    ctx->stamp += (uint32_t)hctl.levels + 3;

    if (materialize) {
      Chunk c;
      c.n_lanes = n_lanes;
      c.rows = total;
      if (bits_req) {
        if ((rc = pick_bit_lanes(ctx, *bits_req, off, segs, n, c))) {
          free_chunk(ctx, c);
          dfree(ctx, cnt, ncnt);
          dfree(ctx, off, ncnt);
          dfree(ctx, tmp, tmpw);
          return rc;
        }
        ep.lane_slot = c.lane_slot;
        ep.bits = c.bits;
        ep.bwords = c.bwords;
        ep.keep_lists = c.lists_kept ? 1u : 0u;
        if (c.bits && !c.lists_kept) {
          // bitset rows are not listed: offsets of the listed rows only
          u64 listed = 0;
          CK(launch_zero_lane_counts(cnt, segs, n_lanes, c.lane_slot, ctx->stream));
          CK(exclusive_scan_u32_to_u64(cnt, off, ncnt, ctx->small + 2, tmp, ctx->stream));
          CK(cudaMemcpyAsync(&listed, ctx->small + 2, 8, cudaMemcpyDeviceToHost, ctx->stream));
          CK(cudaStreamSynchronize(ctx->stream));
          c.rows = listed;
          res->stats.launches += 2;
        }
      }
      if ((rc = dalloc(ctx, &c.lanesrc, n_lanes)) || (rc = dalloc(ctx, &c.lane_off, (uint64_t)n_lanes + 1)) ||
          (rc = dalloc(ctx, &c.dst, c.rows))) {
        free_chunk(ctx, c);
        dfree(ctx, cnt, ncnt);
        dfree(ctx, off, ncnt);
        dfree(ctx, tmp, tmpw);
        return rc;
      }
      ep.dst = c.dst;
      CK(launch_emit(nw, true, false, ep, ctx->stream));
      CK(launch_gather_lane_off(off, segs, n_lanes, ctx->small + 2, c.lane_off, ctx->stream));
      CK(cudaMemcpyAsync(c.lanesrc, w.lanesrc, n_lanes * 4, cudaMemcpyDeviceToDevice, ctx->stream));
      // digest of the written rows (a block per source lane)
      CK(launch_row_digest(w.lanesrc, c.lane_off, n_lanes, c.dst, ctx->small, ctx->stream));
      res->chunks.push_back(c);
      CK(rb_queue(ctx, RB_SMALL, ctx->small, 16));
      res->stats.launches += 4;
    }
    CK(cudaEventRecord(ctx->ev[3], ctx->stream));
    dfree(ctx, cnt, ncnt);
    dfree(ctx, off, ncnt);
    dfree(ctx, tmp, tmpw);
    CK(cudaEventSynchronize(ctx->ev[3]));
    CK(cudaStreamSynchronize(ctx->stream));
    if (materialize) std::memcpy(hdig, ctx->rb_host + RB_SMALL, 16);
    res->dsum += hdig[0];
    res->dxor ^= hdig[1];
    float ms_bfs = 0, ms_emit = 0;
    cudaEventElapsedTime(&ms_bfs, ctx->ev[0], ctx->ev[1]);
    cudaEventElapsedTime(&ms_emit, ctx->ev[2], ctx->ev[3]);
    s.bfs_ms += ms_bfs;
    s.emit_ms += ms_emit;
  }
  return RPQ_OK;
}

int check_rpq_flags(rpq_ctx *ctx, uint32_t flags) {
  uint32_t mode = flags & (RPQ_MATERIALIZE | RPQ_COUNT_ONLY);
  if (mode != RPQ_MATERIALIZE && mode != RPQ_COUNT_ONLY)
    return set_err(ctx, RPQ_ERR_INVALID_ARG, "flags need exactly one of RPQ_MATERIALIZE, RPQ_COUNT_ONLY");
  if ((flags & RPQ_FORCE_PUSH) && (flags & RPQ_FORCE_PULL))
    return set_err(ctx, RPQ_ERR_INVALID_ARG, "RPQ_FORCE_PUSH and RPQ_FORCE_PULL are exclusive");
  if (flags & ~(RPQ_MATERIALIZE | RPQ_COUNT_ONLY | RPQ_REVERSE | RPQ_FORCE_PUSH | RPQ_FORCE_PULL))
    return set_err(ctx, RPQ_ERR_INVALID_ARG, "unknown flag bits");
  return RPQ_OK;
}

int run_sources(rpq_ctx *ctx, const rpq_graph *g, const rpq_query *q, std::vector<uint32_t> &srcs, uint32_t flags,
                rpq_result **out) {
  rpq_result *r = new rpq_result;
  r->ctx = ctx;
  ctx->live++;
  r->arity = 2;
  r->materialized = (flags & RPQ_MATERIALIZE) != 0;
  std::memset(&r->stats, 0, sizeof(r->stats));
  int rc = eval_rpq(ctx, g, q, srcs, flags, r);
  if (rc) {
    free_result(r);
    return rc;
  }
  *out = r;
  return RPQ_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int rpq_create(rpq_ctx **out, int device, uint64_t mem_budget_bytes, void *cuda_stream) {
  if (!out) {
    g_create_error = "out is NULL";
    return RPQ_ERR_INVALID_ARG;
  }
  *out = nullptr;
  rpq_ctx *c = new rpq_ctx;
  c->device = device;
  if (device < 0) {
    *out = c;
    return RPQ_OK;
  }
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaFree(0);
  size_t free_b = 0, total_b = 0;
  if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
  if (e != cudaSuccess) {
    g_create_error = std::string("CUDA device unavailable: ") + cudaGetErrorString(e);
    delete c;
    return RPQ_ERR_CUDA;
  }
  c->stream = (cudaStream_t)cuda_stream;
  c->budget = mem_budget_bytes ? mem_budget_bytes : (uint64_t)(free_b * 0.9);
  {
    // Per-launch buffers (emission counts, result rows) come and go every
    // launch; a pool that keeps freed memory mapped makes those allocations
    // free of page-mapping work.  The pool never holds more than the peak the
    // budget allowed, and it is released with the context.
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (cudaMemPoolCreate(&c->pool, &props) == cudaSuccess) {
      uint64_t keep = ~0ull;
      cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    } else {
      c->pool = nullptr;
      cudaGetLastError();
    }
  }
  for (int i = 0; i < 4; i++) cudaEventCreate(&c->ev[i]);
  if (msbfs_max_blocks(1, BFS_THREADS_HOST, &c->bpsm[0], &c->sms) || msbfs_max_blocks(4, BFS_THREADS_HOST, &c->bpsm[1], &c->sms)) {
    g_create_error = "occupancy query failed";
    rpq_destroy(c);
    return RPQ_ERR_CUDA;
  }
  if (const char *a = std::getenv("RPQ_ALPHA")) c->alpha = (float)std::atof(a);
  if (const char *m = std::getenv("RPQ_MAX_GROUPS")) c->max_groups = (uint32_t)std::min(16, std::max(1, std::atoi(m)));
  if (const char *t = std::getenv("RPQ_TRACE")) c->trace = std::atoi(t) != 0;
  if (const char *sc = std::getenv("RPQ_SPILL_CAP")) {
    c->spill_cap = (uint64_t)std::min<long long>((long long)SPILL_CAP, std::max(0ll, std::atoll(sc)));
    c->batch.spill_cap = c->spill_cap;
  }
  if (const char *b = std::getenv("RPQ_BATCH_LIST_CAP"))
    c->batch.list_cap = (uint64_t)std::max(1024ll, std::atoll(b));
  if (dalloc(c, &c->ctl, 1) || dalloc(c, &c->small, 8)) {
    g_create_error = c->err;
    rpq_destroy(c);
    return RPQ_ERR_CUDA;
  }
  {
    // run_rpq_static's array is reserved here, not at its first call
    std::string msg;
    if (static_scratch_prepare(&c->static_scratch, &msg) != RPQ_OK) {
      g_create_error = msg;
      rpq_destroy(c);
      return RPQ_ERR_CUDA;
    }
  }
  *out = c;
  return RPQ_OK;
}

}  // extern "C"

namespace {

void destroy_now(rpq_ctx *c) {
  if (c->device >= 0) {
    cudaSetDevice(c->device);
    free_workspace(c);
    dfree(c, c->ctl, 1);
    dfree(c, c->small, 8);
    cudaStreamSynchronize(c->stream);
    for (int i = 0; i < 4; i++)
      if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    for (rpq_ctx *h : c->helpers) rpq_destroy(h);
    for (cudaStream_t hs : c->helper_streams) cudaStreamDestroy(hs);
    if (c->pool) cudaMemPoolDestroy(c->pool);
    for (void *h : c->pinned) cudaFreeHost(h);
    if (c->rb_host) cudaFreeHost(c->rb_host);
  }
  delete c;
}

// A graph or result was freed; finish a deferred rpq_destroy.
void release_handle(rpq_ctx *c) {
  c->live--;
  if (c->closing && c->live <= 0) destroy_now(c);
}

}  // namespace

extern "C" {

void rpq_destroy(rpq_ctx *c) {
  if (!c) return;
  c->closing = true;
  if (c->live <= 0) destroy_now(c);
}

const char *rpq_last_error(const rpq_ctx *c) { return c ? c->err.c_str() : g_create_error.c_str(); }

int rpq_set_stream(rpq_ctx *ctx, void *stream) {
  if (!ctx) return RPQ_ERR_INVALID_ARG;
  if (!usable(ctx)) return RPQ_ERR_NO_DEVICE;
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->stream = (cudaStream_t)stream;
  return RPQ_OK;
}

int rpq_set_option(rpq_ctx *ctx, const char *name, double value) {
  if (!ctx || !name) return set_err(ctx, RPQ_ERR_INVALID_ARG, "null argument");
  const std::string n(name);
  if (n == "alpha" && value > 0) {
    ctx->alpha = (float)value;
  } else if (n == "lane_alpha" && value > 0) {
    ctx->lane_alpha = (float)value;
  } else if (n == "pull_dynamic" && (value == 0 || value == 1)) {
    ctx->pull_dynamic = value != 0 ? 1u : 0u;
  } else if (n == "lane_by_source" && (value == 0 || value == 1)) {
    ctx->lane_by_source = value != 0 ? 1u : 0u;
  } else if (n == "crpq_bitset_frac" && value >= 0 && value <= 2) {
    ctx->crpq_bitset_frac = value;
  } else if (n == "grid_share" && value > 0 && value <= 1) {
    ctx->grid_share = value;
  } else if (n == "max_groups" && value >= 1 && value <= 16) {
    ctx->max_groups = (uint32_t)value;
  } else if (n == "time_limit_s" && value > 0) {
    ctx->time_limit_ns = (uint64_t)(value * 1e9);
  } else if (n == "batch_evict" && value >= 0) {
    ctx->batch.evict_at = (uint64_t)value;
  } else if (n == "batch_multi" && (value == 0 || value == 1)) {
    ctx->batch.multi = value != 0;
  } else if (n == "batch_streams" && value >= 1 && value <= 16) {
    ctx->batch.streams = (uint32_t)value;
  } else if (n == "batch_lanes" && value >= 0 && value <= 4096) {
    ctx->batch.lanes = (uint32_t)value;
  } else if (n == "batch_direct" && (value == 0 || value == 1)) {
    ctx->batch.direct = value != 0;
  } else if (n == "batch_hash" && (value == 0 || value == 1)) {
    ctx->batch.hash = value != 0;
  } else {
    return set_err(ctx, RPQ_ERR_INVALID_ARG, "unknown option or value out of range: " + n);
  }
  return RPQ_OK;
}

int rpq_get_option(const rpq_ctx *ctx, const char *name, double *value) {
  if (!ctx || !name || !value) return RPQ_ERR_INVALID_ARG;
  const std::string n(name);
  if (n == "alpha")
    *value = ctx->alpha;
  else if (n == "lane_alpha")
    *value = ctx->lane_alpha;
  else if (n == "pull_dynamic")
    *value = ctx->pull_dynamic;
  else if (n == "lane_by_source")
    *value = ctx->lane_by_source;
  else if (n == "crpq_bitset_frac")
    *value = ctx->crpq_bitset_frac;
  else if (n == "grid_share")
    *value = ctx->grid_share;
  else if (n == "max_groups")
    *value = ctx->max_groups;
  else if (n == "time_limit_s")
    *value = ctx->time_limit_ns * 1e-9;
  else if (n == "batch_evict")
    *value = (double)ctx->batch.evict_at;
  else if (n == "batch_threads")
    *value = ctx->batch.threads;
  else if (n == "batch_queries_per_launch")
    *value = ctx->batch.queries_per_launch;
  else if (n == "batch_multi")
    *value = ctx->batch.multi ? 1 : 0;
  else if (n == "batch_streams")
    *value = ctx->batch.streams;
  else if (n == "batch_lanes")
    *value = ctx->batch.lanes;
  else if (n == "batch_direct")
    *value = ctx->batch.direct ? 1 : 0;
  else if (n == "batch_hash")
    *value = ctx->batch.hash ? 1 : 0;
  else
    return RPQ_ERR_INVALID_ARG;
  return RPQ_OK;
}

int load_graph(rpq_ctx *ctx, uint32_t n_vertices, uint32_t n_labels, uint64_t n_edges, const uint32_t *src,
               const uint32_t *dst, const uint16_t *label, const uint8_t *vertex_label, rpq_graph **out) {
  if (!ctx || !out) return set_err(ctx, RPQ_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (!usable(ctx)) return RPQ_ERR_NO_DEVICE;
  if (n_edges && (!src || !dst || !label)) return set_err(ctx, RPQ_ERR_INVALID_ARG, "null edge array");
  if (n_vertices == 0 || n_vertices >= (1u << 31)) return set_err(ctx, RPQ_ERR_INVALID_ARG, "bad n_vertices");
  if (n_labels == 0 || n_labels > RPQ_MAX_LABELS) return set_err(ctx, RPQ_ERR_INVALID_ARG, "bad n_labels");
  if (n_edges >= (1ull << 32)) return set_err(ctx, RPQ_ERR_INVALID_ARG, "n_edges must be < 2^32");
  if (graph_key_bits(n_vertices, n_labels) > 64)
    return set_err(ctx, RPQ_ERR_INVALID_ARG, "graph too large for 64-bit edge keys");
  rpq_graph *gr = new rpq_graph;
  gr->ctx = ctx;
  ctx->live++;
  uint32_t *d_src = nullptr, *d_dst = nullptr;
  uint16_t *d_lab = nullptr;
  int rc = RPQ_OK;
  const uint64_t m = n_edges;
  const uint64_t rows = (uint64_t)n_labels * (n_vertices + 1);
  // the graph arrays: 2 offset arrays + 2 column arrays (+ vertex labels)
  const uint64_t gbytes = rows * 8 + m * 8 + (vertex_label ? n_vertices : 0);
  // sort scratch (keys x3, flags, histograms) comes from the same budget
  const uint64_t scratch = m * 30 + (64ull << 20);
  if (ctx->used + gbytes + scratch + m * 10 > ctx->budget) {
    delete gr;
    release_handle(ctx);
    return set_err(ctx, RPQ_ERR_OUT_OF_BUDGET, "graph does not fit the device memory budget");
  }
  cudaStream_t st = ctx->stream;
  std::string msg;
  if ((rc = dalloc(ctx, &d_src, m)) || (rc = dalloc(ctx, &d_dst, m)) || (rc = dalloc(ctx, &d_lab, m))) goto fail;
  if (m) {
    cudaError_t e;
    if ((e = cudaMemcpyAsync(d_src, src, m * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d_dst, dst, m * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d_lab, label, m * 2, cudaMemcpyHostToDevice, st)) != cudaSuccess) {
      rc = cuda_err(ctx, e, "cudaMemcpyAsync");
      goto fail;
    }
  }
  rc = build_graph(&gr->g, n_vertices, n_labels, m, d_src, d_dst, d_lab, st, &msg);
  if (rc) {
    set_err(ctx, rc, msg);
    goto fail;
  }
  if (vertex_label) {
    rc = dalloc(ctx, &gr->g.vlabel, n_vertices);
    if (rc) goto fail;
    gr->g.vlabel_host.assign(vertex_label, vertex_label + n_vertices);
    cudaError_t e = cudaMemcpyAsync(gr->g.vlabel, vertex_label, n_vertices, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
      rc = cuda_err(ctx, e, "cudaMemcpyAsync");
      goto fail;
    }
  }
  {
    // the graph arrays were allocated inside build_graph outside the budget
    // accounting; account for them now
    uint64_t b = rows * 8 + gr->g.m * 8 +
                 12ull * ((uint64_t)gr->g.hchunk_in_off.back() + gr->g.hchunk_out_off.back());
    ctx->used += b;
    gr->bytes = b;
  }
  dfree(ctx, d_src, m);
  dfree(ctx, d_dst, m);
  dfree(ctx, d_lab, m);
  {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      rc = cuda_err(ctx, e, "load_graph");
      free_graph(gr);
      return rc;
    }
  }
  *out = gr;
  return RPQ_OK;
fail:
  dfree(ctx, d_src, m);
  dfree(ctx, d_dst, m);
  dfree(ctx, d_lab, m);
  if (gr->g.out_off) cudaFreeAsync(gr->g.out_off, st);
  if (gr->g.in_off) cudaFreeAsync(gr->g.in_off, st);
  if (gr->g.out_col) cudaFreeAsync(gr->g.out_col, st);
  if (gr->g.in_col) cudaFreeAsync(gr->g.in_col, st);
  if (gr->g.hchunk_in) cudaFreeAsync(gr->g.hchunk_in, st);
  if (gr->g.hchunk_out) cudaFreeAsync(gr->g.hchunk_out, st);
  if (gr->g.vlabel) dfree(ctx, gr->g.vlabel, n_vertices);
  delete gr;
  release_handle(ctx);
  return rc;
}

int graph_info(const rpq_graph *g, uint32_t *n_vertices, uint32_t *n_labels, uint64_t *n_edges) {
  if (!g) return RPQ_ERR_INVALID_ARG;
  if (n_vertices) *n_vertices = g->g.n;
  if (n_labels) *n_labels = g->g.L;
  if (n_edges) *n_edges = g->g.m;
  return RPQ_OK;
}

void free_graph(rpq_graph *g) {
  if (!g) return;
  rpq_ctx *ctx = g->ctx;
  cudaSetDevice(ctx->device);
  cudaStream_t st = ctx->stream;
  cudaFreeAsync(g->g.out_off, st);
  cudaFreeAsync(g->g.in_off, st);
  cudaFreeAsync(g->g.out_col, st);
  cudaFreeAsync(g->g.in_col, st);
  cudaFreeAsync(g->g.hchunk_in, st);
  cudaFreeAsync(g->g.hchunk_out, st);
  ctx->used -= std::min(ctx->used, g->bytes);
  if (g->g.vlabel) dfree(ctx, g->g.vlabel, g->g.n);
  delete g;
  release_handle(ctx);
}

int compile_rpq(rpq_ctx *ctx, const char *regex, const char *const *label_names, uint32_t n_names,
                rpq_query **out) {
  if (!ctx || !out || !regex) return set_err(ctx, RPQ_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (label_names == nullptr && n_names != 0) return set_err(ctx, RPQ_ERR_INVALID_ARG, "names NULL but n_names > 0");
  rpq_query *q = new rpq_query;
  std::string msg;
  int rc = compile_regex(regex, label_names, n_names, &q->hq, &msg);
  if (rc) {
    delete q;
    return set_err(ctx, rc, msg);
  }
  *out = q;
  return RPQ_OK;
}

int query_info(const rpq_query *q, uint32_t *n_states, uint32_t *n_labels_out, uint64_t *final_mask, int32_t *next) {
  if (!q) return RPQ_ERR_INVALID_ARG;
  if (n_states) *n_states = q->hq.d.n_states;
  if (n_labels_out) *n_labels_out = q->hq.d.n_labels;
  if (final_mask) *final_mask = q->hq.d.final_mask;
  if (next && !q->hq.next.empty()) std::memcpy(next, q->hq.next.data(), q->hq.next.size() * 4);
  return RPQ_OK;
}

void free_query(rpq_query *q) { delete q; }

int run_rpq(rpq_ctx *ctx, const rpq_graph *g, const rpq_query *q, const uint32_t *sources, uint32_t n_sources,
            uint32_t flags, rpq_result **out) {
  if (!ctx || !g || !q || !out) return set_err(ctx, RPQ_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (!usable(ctx)) return RPQ_ERR_NO_DEVICE;
  int rc = check_rpq_flags(ctx, flags);
  if (rc) return rc;
  if (!sources && n_sources) return set_err(ctx, RPQ_ERR_INVALID_ARG, "sources NULL but n_sources > 0");
  std::vector<uint32_t> srcs;
  if (!sources) {
    srcs.resize(g->g.n);
    for (uint32_t v = 0; v < g->g.n; v++) srcs[v] = v;
  } else {
    srcs.assign(sources, sources + n_sources);
    for (uint32_t s : srcs)
      if (s >= g->g.n) return set_err(ctx, RPQ_ERR_INVALID_ARG, "source id out of range");
    std::sort(srcs.begin(), srcs.end());
    srcs.erase(std::unique(srcs.begin(), srcs.end()), srcs.end());
  }
  return run_sources(ctx, g, q, srcs, flags, out);
}

int run_rpq_range(rpq_ctx *ctx, const rpq_graph *g, const rpq_query *q, uint32_t src_begin, uint32_t src_end,
                  uint32_t flags, rpq_result **out) {
  if (!ctx || !g || !q || !out) return set_err(ctx, RPQ_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (!usable(ctx)) return RPQ_ERR_NO_DEVICE;
  int rc = check_rpq_flags(ctx, flags);
  if (rc) return rc;
  if (src_begin > src_end || src_end > g->g.n) return set_err(ctx, RPQ_ERR_INVALID_ARG, "bad source range");
  std::vector<uint32_t> srcs(src_end - src_begin);
  for (uint32_t i = 0; i < srcs.size(); i++) srcs[i] = src_begin + i;
  return run_sources(ctx, g, q, srcs, flags, out);
}

int run_rpq_middle(rpq_ctx *ctx, const rpq_graph *gr, const rpq_query *alpha, const rpq_query *beta,
                   const uint32_t *sources, uint32_t n_sources, uint32_t flags, rpq_result **out) {
  if (!ctx || !gr || !alpha || !beta || !out) return set_err(ctx, RPQ_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (!usable(ctx)) return RPQ_ERR_NO_DEVICE;
  int rc = check_rpq_flags(ctx, flags);
  if (rc) return rc;
  if (flags & RPQ_REVERSE) return set_err(ctx, RPQ_ERR_INVALID_ARG, "RPQ_REVERSE is not a start-in-the-middle flag");
  if (!sources && n_sources) return set_err(ctx, RPQ_ERR_INVALID_ARG, "sources NULL but n_sources > 0");
  const DevGraph &g = gr->g;
  const uint32_t n = g.n;
  std::vector<uint32_t> srcs;
  if (!sources) {
    srcs.resize(n);
    for (uint32_t v = 0; v < n; v++) srcs[v] = v;
  } else {
    srcs.assign(sources, sources + n_sources);
    for (uint32_t s : srcs)
      if (s >= n) return set_err(ctx, RPQ_ERR_INVALID_ARG, "source id out of range");
    std::sort(srcs.begin(), srcs.end());
    srcs.erase(std::unique(srcs.begin(), srcs.end()), srcs.end());
  }
  const HostQuery &ha = alpha->hq;
  // the label X of the materialized pairs: above the graph's labels and alpha's
  const uint32_t X = std::max(g.L, ha.d.n_labels);
  if (X >= RPQ_MAX_LABELS) return set_err(ctx, RPQ_ERR_TOO_COMPLEX, "no label id left for the materialized pairs");
  rpq_query qx;
  {
    std::string msg;
    if ((rc = dfa_then_label(ha, X, &qx.hq, &msg))) return set_err(ctx, rc, msg);
  }
  rpq_result *res = new rpq_result;
  res->ctx = ctx;
  ctx->live++;
  res->arity = 2;
  res->materialized = (flags & RPQ_MATERIALIZE) != 0;
  std::memset(&res->stats, 0, sizeof(res->stats));
  cudaStream_t st = ctx->stream;
  // 1. where alpha paths can end: every vertex when alpha accepts the empty
  //    word, else the vertices with an in-edge on a label entering an
  //    accepting state of alpha
  std::vector<uint32_t> mid;
  if (ha.d.n_states && (ha.d.final_mask & 1u)) {
    mid.resize(n);
    for (uint32_t v = 0; v < n; v++) mid[v] = v;
  } else if (ha.d.n_states) {
    unsigned long long lmask = 0;
    for (uint32_t q = 0; q < ha.d.n_states; q++)
      for (uint32_t l = 0; l < ha.d.n_labels && l < g.L; l++) {
        const int32_t t = ha.next[(size_t)q * ha.d.n_labels + l];
        if (t >= 0 && ((ha.d.final_mask >> t) & 1u)) lmask |= 1ull << l;
      }
    if (lmask) {
      u32 *dall = nullptr;
      unsigned char *dflag = nullptr;
      std::vector<uint32_t> all(n);
      for (uint32_t v = 0; v < n; v++) all[v] = v;
      std::vector<unsigned char> flag(n);
      if ((rc = dalloc(ctx, &dall, n)) || (rc = dalloc(ctx, &dflag, n))) {
        dfree(ctx, dall, n);
        free_result(res);
        return rc;
      }
      cudaError_t e = cudaMemcpyAsync(dall, all.data(), 4ull * n, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = launch_source_filter(g.in_off, n, g.L, lmask, dall, n, dflag, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(flag.data(), dflag, n, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      dfree(ctx, dall, n);
      dfree(ctx, dflag, n);
      if (e != cudaSuccess) {
        free_result(res);
        return cuda_err(ctx, e, "middle vertices");
      }
      for (uint32_t v = 0; v < n; v++)
        if (flag[v]) mid.push_back(v);
    }
  }
  // 2. R(beta) from those vertices, materialized per start vertex
  std::vector<RowChunk> chunks;
  rpq_stats bst;
  std::memset(&bst, 0, sizeof(bst));
  if (!mid.empty() && (rc = rpq_rows_for_sources(ctx, gr, beta, mid, false, &chunks, &bst))) {
    for (RowChunk &c : chunks) free_row_chunk(ctx, c);
    free_result(res);
    return rc;
  }
  uint64_t R = 0;
  for (const RowChunk &c : chunks) R += c.rows;
  // 3. a temporary graph: G's edges plus the pairs of R(beta) as label X
  const uint64_t m2 = g.m + R;
  if (m2 >= (1ull << 32)) {
    for (RowChunk &c : chunks) free_row_chunk(ctx, c);
    free_result(res);
    return set_err(ctx, RPQ_ERR_TOO_COMPLEX, "the materialized pairs and the graph exceed 2^32 edges");
  }
  rpq_graph g2;
  g2.ctx = ctx;
  u32 *d_src = nullptr, *d_dst = nullptr;
  uint16_t *d_lab = nullptr;
  if ((rc = dalloc(ctx, &d_src, m2)) || (rc = dalloc(ctx, &d_dst, m2)) || (rc = dalloc(ctx, &d_lab, m2))) {
    dfree(ctx, d_src, m2);
    dfree(ctx, d_dst, m2);
    for (RowChunk &c : chunks) free_row_chunk(ctx, c);
    free_result(res);
    return rc;
  }
  cudaError_t e = launch_csr_triples(g.out_off, g.out_col, n, g.L, d_src, d_dst, d_lab, st);
  uint64_t base = g.m;
  for (const RowChunk &c : chunks) {
    if (e == cudaSuccess)
      e = launch_chunk_triples(c.lanesrc, c.lane_off, c.n_lanes, c.dst, base, (uint16_t)X, d_src, d_dst, d_lab, st);
    base += c.rows;
  }
  for (RowChunk &c : chunks) free_row_chunk(ctx, c);
  std::string msg;
  if (e == cudaSuccess) {
    rc = build_graph(&g2.g, n, X + 1, m2, d_src, d_dst, d_lab, st, &msg);
    if (rc) set_err(ctx, rc, msg);
  } else {
    rc = cuda_err(ctx, e, "middle-plan edge list");
  }
  dfree(ctx, d_src, m2);
  dfree(ctx, d_dst, m2);
  dfree(ctx, d_lab, m2);
  // 4. alpha . X over the temporary graph, from the requested start vertices
  if (rc == RPQ_OK) rc = eval_rpq(ctx, &g2, &qx, srcs, flags, res);
  if (g2.g.out_off) cudaFreeAsync(g2.g.out_off, st);
  if (g2.g.in_off) cudaFreeAsync(g2.g.in_off, st);
  if (g2.g.out_col) cudaFreeAsync(g2.g.out_col, st);
  if (g2.g.in_col) cudaFreeAsync(g2.g.in_col, st);
  if (g2.g.hchunk_in) cudaFreeAsync(g2.g.hchunk_in, st);
  if (g2.g.hchunk_out) cudaFreeAsync(g2.g.hchunk_out, st);
  if (rc) {
    free_result(res);
    return rc;
  }
  // the plan's work: the materialization and the final traversal
  rpq_stats &s2 = res->stats;
  s2.product_edges += bst.product_edges;
  s2.product_vertices += bst.product_vertices;
  s2.levels += bst.levels;
  s2.push_levels += bst.push_levels;
  s2.pull_levels += bst.pull_levels;
  s2.bfs_ms += bst.bfs_ms;
  s2.emit_ms += bst.emit_ms;
  s2.bfs_launches += bst.bfs_launches;
  s2.launches += bst.launches + 2 + chunks.size();
  s2.alg_bytes += bst.alg_bytes;
  *out = res;
  return RPQ_OK;
}

int run_crpq(rpq_ctx *ctx, const rpq_graph *g, uint32_t n_vars, const int32_t *var_label, const crpq_atom *atoms,
             uint32_t n_atoms, const uint32_t *restrict0, uint32_t n_restrict0, uint32_t flags, rpq_result **out) {
  if (!ctx || !g || !atoms || !out) return set_err(ctx, RPQ_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (!usable(ctx)) return RPQ_ERR_NO_DEVICE;
  int rc = check_rpq_flags(ctx, flags);
  if (rc) return rc;
  return crpq_eval(ctx, g, n_vars, var_label, atoms, n_atoms, restrict0, n_restrict0, flags, out);
}

int run_rpq_batch(rpq_ctx *ctx, const rpq_graph *g, uint32_t n_queries, const rpq_query *const *queries,
                  const uint32_t *sources, uint32_t flags, rpq_result **out) {
  if (!ctx || !g || !out || (n_queries && (!queries || !sources)))
    return set_err(ctx, RPQ_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (!usable(ctx)) return RPQ_ERR_NO_DEVICE;
  const bool per_query = (flags & RPQ_PER_QUERY) != 0;
  if (per_query) flags = (flags & ~(uint32_t)RPQ_PER_QUERY) | RPQ_COUNT_ONLY;
  uint32_t mode = flags & (RPQ_MATERIALIZE | RPQ_COUNT_ONLY);
  if ((mode != RPQ_MATERIALIZE && mode != RPQ_COUNT_ONLY) || (flags & ~(RPQ_MATERIALIZE | RPQ_COUNT_ONLY)))
    return set_err(ctx, RPQ_ERR_INVALID_ARG,
                   "run_rpq_batch takes RPQ_MATERIALIZE, RPQ_COUNT_ONLY or RPQ_PER_QUERY (alone)");
  for (uint32_t i = 0; i < n_queries; i++) {
    if (!queries[i]) return set_err(ctx, RPQ_ERR_INVALID_ARG, "null query");
    if (sources[i] >= g->g.n) return set_err(ctx, RPQ_ERR_INVALID_ARG, "source id out of range");
  }
  const bool materialize = mode == RPQ_MATERIALIZE;
  BatchOut bo;
  bo.per_query = per_query;
  int rc = n_queries ? batch_run(ctx, g, n_queries, queries, sources, materialize, ctx->batch, &bo) : RPQ_OK;
  auto drop = [&]() {
    for (auto &c : bo.chunks) dev_free(ctx, c.first, c.second * 8);
    bo.chunks.clear();
  };
  if (rc) {
    drop();
    return rc;
  }
  u32 *tuples = nullptr;
  if (materialize && bo.count) {
    if (bo.chunks.size() == 1) {
      tuples = bo.chunks[0].first;
      bo.chunks.clear();
    } else {
      if ((rc = dev_alloc(ctx, (void **)&tuples, bo.count * 8))) {
        drop();
        return rc;
      }
      uint64_t o = 0;
      for (auto &c : bo.chunks) {
        cudaMemcpyAsync(tuples + 2 * o, c.first, c.second * 8, cudaMemcpyDeviceToDevice, ctx->stream);
        o += c.second;
      }
      drop();
    }
  }
  bo.stats.lane_words = 0;
  rc = make_tuple_result(ctx, 2, tuples, bo.count, bo.dsum, bo.dxor, materialize, bo.stats, out);
  if (rc == RPQ_OK && per_query) {
    (*out)->qstats.swap(bo.qstats);
    (*out)->qdone_ms.swap(bo.qdone_ms);
  }
  return rc;
}

int rpq_autotune_batch(rpq_ctx *ctx, const rpq_graph *g, uint32_t n_queries, const rpq_query *const *queries,
                       const uint32_t *sources, uint32_t *threads_out, uint32_t *queries_per_launch_out) {
  if (!ctx || !g || (n_queries && (!queries || !sources))) return set_err(ctx, RPQ_ERR_INVALID_ARG, "null argument");
  if (!usable(ctx)) return RPQ_ERR_NO_DEVICE;
  for (uint32_t i = 0; i < n_queries; i++)
    if (!queries[i] || sources[i] >= g->g.n) return set_err(ctx, RPQ_ERR_INVALID_ARG, "bad query or source");
  const uint32_t sample = std::min<uint32_t>(n_queries, 1024);
  BatchTuning best = ctx->batch;
  double best_s = -1;
  // Candidates: every query straight to lane-mode launches, or a shared
  // per-query launch first (visited set: dense bitmaps or hash tables; block
  // size; eviction threshold) with the evicted queries in lane-mode launches.
  // (Never evicting is not a candidate: a sample that keeps its heavy queries
  // in the shared launch says little about a full batch that would not.)
  std::vector<BatchTuning> cands;
  {
    BatchTuning c = ctx->batch;
    c.direct = true;
    if (c.lanes == 0) c.lanes = 4096;
    cands.push_back(c);
  }
  for (int hash = 0; hash < 2; hash++)
    for (int t : {256, 512})
      for (uint64_t ev : {1ull << 10, 1ull << 12, 1ull << 14}) {
        BatchTuning c = ctx->batch;
        c.direct = false;
        if (c.lanes == 0) c.lanes = 4096;
        c.hash = hash != 0;
        c.threads = t;
        c.evict_at = ev;
        cands.push_back(c);
      }
  for (const BatchTuning &cand : cands) {
    BatchOut bo;
    bo.per_query = true;
    cudaStreamSynchronize(ctx->stream);
    auto t0 = std::chrono::steady_clock::now();
    int rc = sample ? batch_run(ctx, g, sample, queries, sources, false, cand, &bo) : RPQ_OK;
    cudaStreamSynchronize(ctx->stream);
    double s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (rc) return rc;
    if (best_s < 0 || s < best_s) {
      best_s = s;
      best = cand;
    }
  }
  ctx->batch = best;
  if (threads_out) *threads_out = (uint32_t)best.threads;
  if (queries_per_launch_out) *queries_per_launch_out = best.queries_per_launch;
  return RPQ_OK;
}

int result_info(const rpq_result *r, uint64_t *count, uint32_t *arity, uint64_t *digest_sum, uint64_t *digest_xor) {
  if (!r) return RPQ_ERR_INVALID_ARG;
  if (count) *count = r->count;
  if (arity) *arity = r->arity;
  if (digest_sum) *digest_sum = r->dsum;
  if (digest_xor) *digest_xor = r->dxor;
  return RPQ_OK;
}

int result_query_stats(const rpq_result *r, uint32_t i, uint64_t *count, uint64_t *digest_sum, uint64_t *digest_xor) {
  if (!r || 3ull * i + 2 >= r->qstats.size()) return RPQ_ERR_INVALID_ARG;
  if (count) *count = r->qstats[3ull * i];
  if (digest_sum) *digest_sum = r->qstats[3ull * i + 1];
  if (digest_xor) *digest_xor = r->qstats[3ull * i + 2];
  return RPQ_OK;
}

int result_query_time(const rpq_result *r, uint32_t i, double *ms) {
  if (!r || !ms || i >= r->qdone_ms.size()) return RPQ_ERR_INVALID_ARG;
  *ms = r->qdone_ms[i];
  return RPQ_OK;
}

int result_stats(const rpq_result *r, rpq_stats *out) {
  if (!r || !out) return RPQ_ERR_INVALID_ARG;
  *out = r->stats;
  return RPQ_OK;
}

int fetch_pairs(const rpq_result *r, uint64_t offset, uint64_t max_rows, uint32_t *out, uint64_t *n_rows) {
  if (!r || (!out && max_rows) || !n_rows) return set_err(r ? r->ctx : nullptr, RPQ_ERR_INVALID_ARG, "null argument");
  rpq_ctx *ctx = r->ctx;
  *n_rows = 0;
  if (!r->materialized) return set_err(ctx, RPQ_ERR_INVALID_ARG, "result was made with RPQ_COUNT_ONLY");
  if (offset >= r->count || max_rows == 0) return RPQ_OK;
  cudaSetDevice(ctx->device);
  const uint64_t want = std::min<uint64_t>(max_rows, r->count - offset);
  if (r->arity != 2 || r->tuples) {
    CK(cudaMemcpyAsync(out, r->tuples + offset * r->arity, want * r->arity * 4, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    *n_rows = want;
    return RPQ_OK;
  }
  const uint64_t piece = 1ull << 24;
  u32 *stage = nullptr;
  int rc = dalloc(ctx, &stage, 2 * std::min(piece, want));
  if (rc) return rc;
  uint64_t done = 0, base = 0;
  for (const Chunk &c : r->chunks) {
    uint64_t c_end = base + c.rows;
    while (done < want && offset + done < c_end) {
      uint64_t first = offset + done - base;
      uint64_t k = std::min<uint64_t>({piece, want - done, c.rows - first});
      cudaError_t e = launch_expand_pairs(c.lanesrc, c.lane_off, c.n_lanes, c.dst, first, k, stage, ctx->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(out + 2 * done, stage, k * 8, cudaMemcpyDeviceToHost, ctx->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
      if (e != cudaSuccess) {
        dfree(ctx, stage, 2 * std::min(piece, want));
        return cuda_err(ctx, e, "fetch_pairs");
      }
      done += k;
    }
    base = c_end;
    if (done >= want) break;
  }
  dfree(ctx, stage, 2 * std::min(piece, want));
  *n_rows = done;
  return RPQ_OK;
}

void free_result(rpq_result *r) {
  if (!r) return;
  rpq_ctx *ctx = r->ctx;
  if (ctx && ctx->device >= 0) {
    cudaSetDevice(ctx->device);
    for (Chunk &c : r->chunks) free_chunk(ctx, c);
    if (r->tuples) dev_free(ctx, r->tuples, r->tuple_bytes);
  }
  delete r;
  if (ctx) release_handle(ctx);
}

}  // extern "C"

// Helpers exported to the CRPQ module (same library).
namespace rpq {

int ctx_alloc(rpq_ctx *ctx, void **p, uint64_t bytes) { return dev_alloc(ctx, p, bytes); }
void ctx_free(rpq_ctx *ctx, void *p, uint64_t bytes) { dev_free(ctx, p, bytes); }
cudaStream_t ctx_stream(rpq_ctx *ctx) { return ctx->stream; }
int ctx_error(rpq_ctx *ctx, int code, const std::string &msg) { return set_err(ctx, code, msg); }
int ctx_device(rpq_ctx *ctx) { return ctx->device; }
int ctx_sm_share(rpq_ctx *ctx) { return std::max(1, (int)(ctx->sms * ctx->grid_share)); }
int ctx_bfs_blocks(rpq_ctx *ctx, int nw) { return ctx_sm_share(ctx) * ctx->bpsm[nw == 1 ? 0 : 1]; }
bool ctx_trace(rpq_ctx *ctx) { return ctx->trace; }
BatchTuning ctx_batch_tuning(rpq_ctx *ctx) { return ctx->batch; }
void ctx_copy_tunables(rpq_ctx *to, const rpq_ctx *from) {
  to->alpha = from->alpha;
  to->lane_alpha = from->lane_alpha;
  to->pull_dynamic = from->pull_dynamic;
  to->lane_by_source = from->lane_by_source;
  to->crpq_bitset_frac = from->crpq_bitset_frac;
  to->time_limit_ns = from->time_limit_ns;
  to->spill_cap = from->spill_cap;
  to->batch = from->batch;
}
int ctx_helpers(rpq_ctx *ctx, int k, std::vector<rpq_ctx *> *out) {
  while ((int)ctx->helpers.size() < k) {
    cudaStream_t hs = nullptr;
    if (cudaStreamCreateWithFlags(&hs, cudaStreamNonBlocking) != cudaSuccess)
      return set_err(ctx, RPQ_ERR_CUDA, "helper stream creation failed");
    rpq_ctx *h = nullptr;
    int rc = rpq_create(&h, ctx->device, ctx->budget / (k + 1), hs);
    if (rc) {
      cudaStreamDestroy(hs);
      return set_err(ctx, rc, "helper context creation failed");
    }
    h->alpha = ctx->alpha;
    h->time_limit_ns = ctx->time_limit_ns;
    h->grid_share = ctx->grid_share / k;
    ctx->helpers.push_back(h);
    ctx->helper_streams.push_back(hs);
  }
  for (int i = 0; i < k; i++) {  // follow the parent's current tunables
    ctx->helpers[i]->grid_share = ctx->grid_share / k;
    ctx->helpers[i]->alpha = ctx->alpha;
    ctx->helpers[i]->time_limit_ns = ctx->time_limit_ns;
    ctx->helpers[i]->spill_cap = ctx->spill_cap;
  }
  out->assign(ctx->helpers.begin(), ctx->helpers.begin() + k);
  return RPQ_OK;
}
int ctx_pinned(rpq_ctx *ctx, int count, size_t bytes, void **out) {
  if (ctx->pinned_bytes < bytes) {
    for (void *h : ctx->pinned) cudaFreeHost(h);
    ctx->pinned.clear();
    ctx->pinned_bytes = bytes;
  }
  while ((int)ctx->pinned.size() < count) {
    void *h = nullptr;
    cudaError_t e = cudaHostAlloc(&h, ctx->pinned_bytes, cudaHostAllocDefault);
    if (e != cudaSuccess) return set_err(ctx, RPQ_ERR_CUDA, std::string("pinned host memory: ") + cudaGetErrorString(e));
    ctx->pinned.push_back(h);
  }
  for (int i = 0; i < count; i++) out[i] = ctx->pinned[i];
  return RPQ_OK;
}
bool ctx_cancelled(rpq_ctx *ctx) { return ctx->cancel.load(std::memory_order_relaxed) != 0; }
void ctx_set_cancel(rpq_ctx *ctx, bool on) { ctx->cancel.store(on ? 1 : 0); }
float ctx_alpha(rpq_ctx *ctx) { return ctx->alpha; }
double ctx_crpq_bitset_frac(rpq_ctx *ctx) { return ctx->crpq_bitset_frac; }
uint64_t ctx_budget_left(rpq_ctx *ctx) { return ctx->used < ctx->budget ? ctx->budget - ctx->used : 0; }
uint64_t ctx_time_limit_ns(rpq_ctx *ctx) { return ctx->time_limit_ns; }
void *ctx_static_scratch(rpq_ctx *ctx) { return ctx->static_scratch; }
void ctx_release_workspace(rpq_ctx *ctx) {
  free_workspace(ctx);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->pool) cudaMemPoolTrimTo(ctx->pool, 0);
}
const DevGraph &graph_dev(const rpq_graph *g) { return g->g; }
const HostQuery &query_host(const rpq_query *q) { return q->hq; }

// Runs an RPQ from the given sorted distinct sources, materialized, and hands
// back the per-lane CSR chunks (ownership passes to the caller).
int rpq_rows_for_sources(rpq_ctx *ctx, const rpq_graph *g, const rpq_query *q, std::vector<uint32_t> &srcs,
                         bool reverse, std::vector<RowChunk> *chunks, rpq_stats *stats, uint64_t *dsum,
                         uint64_t *dxor, const RowBitsReq *bits_req) {
  rpq_result r;
  r.ctx = ctx;
  r.materialized = true;
  std::memset(&r.stats, 0, sizeof(r.stats));
  int rc = eval_rpq(ctx, g, q, srcs, RPQ_MATERIALIZE | (reverse ? RPQ_REVERSE : 0u), &r, nullptr, bits_req);
  if (dsum) *dsum += r.dsum;
  if (dxor) *dxor ^= r.dxor;
  if (stats) {
    stats->product_edges += r.stats.product_edges;
    stats->product_vertices += r.stats.product_vertices;
    stats->levels += r.stats.levels;
    stats->push_levels += r.stats.push_levels;
    stats->pull_levels += r.stats.pull_levels;
    stats->group_edges += r.stats.group_edges;
    stats->group_rows += r.stats.group_rows;
    stats->group_vertices += r.stats.group_vertices;
    stats->pull_edges += r.stats.pull_edges;
    stats->pull_vertices += r.stats.pull_vertices;
    stats->alg_bytes += r.stats.alg_bytes;
    stats->group_product_edges += r.stats.group_product_edges;
    stats->group_label_rows += r.stats.group_label_rows;
    stats->lane_groups += r.stats.lane_groups;
    stats->bfs_ms += r.stats.bfs_ms;
    stats->emit_ms += r.stats.emit_ms;
    stats->bfs_launches += r.stats.bfs_launches;
    stats->launches += r.stats.launches;
  }
  for (Chunk &c : r.chunks) {
    if (rc == RPQ_OK) {
      RowChunk rc_;
      rc_.lanesrc = c.lanesrc;
      rc_.lane_off = c.lane_off;
      rc_.dst = c.dst;
      rc_.rows = c.rows;
      rc_.n_lanes = c.n_lanes;
      rc_.bits = c.bits;
      rc_.lane_slot = c.lane_slot;
      rc_.bwords = c.bwords;
      rc_.n_bits = c.n_bits;
      rc_.lists_kept = c.lists_kept;
      chunks->push_back(rc_);
    } else {
      free_chunk(ctx, c);
    }
  }
  r.chunks.clear();
  return rc;
}

// Count-only evaluation from sorted sources (a repeated source is a lane of
// its own) with each lane's own (rows, digest sum, digest xor) in
// lane_stats[3 * i ..]; counters added to *stats.
int rpq_lane_stats_for_sources(rpq_ctx *ctx, const rpq_graph *g, const rpq_query *q,
                               const std::vector<uint32_t> &srcs, std::vector<uint64_t> *lane_stats,
                               rpq_stats *stats) {
  rpq_result r;
  r.ctx = ctx;
  std::memset(&r.stats, 0, sizeof(r.stats));
  int rc = eval_rpq(ctx, g, q, srcs, RPQ_COUNT_ONLY, &r, lane_stats);
  if (stats) {
    stats->product_edges += r.stats.product_edges;
    stats->product_vertices += r.stats.product_vertices;
    stats->levels += r.stats.levels;
    stats->push_levels += r.stats.push_levels;
    stats->pull_levels += r.stats.pull_levels;
    stats->bfs_ms += r.stats.bfs_ms;
    stats->emit_ms += r.stats.emit_ms;
    stats->bfs_launches += r.stats.bfs_launches;
    stats->launches += r.stats.launches;
    stats->alg_bytes += r.stats.alg_bytes;
    stats->group_product_edges += r.stats.group_product_edges;
    stats->group_label_rows += r.stats.group_label_rows;
  }
  return rc;
}

// Count-only evaluation of up to 16 units in one launch, each unit a lane
// group of its own (one 64-lane word, at most 64 start vertices, repeats
// allowed) running its own automaton.  Per lane (rows, digest sum, digest
// xor) in lane_stats, unit by unit in the units' source order; counters
// added to *stats.  TOO_COMPLEX when the union of the automata needs more
// transition entries than a descriptor holds (the caller then runs the units
// apart).
int rpq_lane_stats_multi(rpq_ctx *ctx, const rpq_graph *gr, const std::vector<MultiUnit> &units,
                         std::vector<uint64_t> *lane_stats, rpq_stats *stats) {
  const DevGraph &g = gr->g;
  const uint32_t G = (uint32_t)units.size();
  size_t total_lanes = 0;
  for (const MultiUnit &u : units) {
    if (u.srcs.size() > 64) return set_err(ctx, RPQ_ERR_INVALID_ARG, "a unit holds at most 64 start vertices");
    total_lanes += u.srcs.size();
  }
  lane_stats->assign(3 * total_lanes, 0);
  if (G == 0 || total_lanes == 0) return RPQ_OK;
  if (G > 16) return set_err(ctx, RPQ_ERR_INVALID_ARG, "at most 16 units per launch");
  const uint32_t n = g.n, L = g.L;
  uint32_t Q = 0;
  for (const MultiUnit &u : units) Q = std::max(Q, query_host(u.q).d.n_states);
  if (Q == 0) return RPQ_OK;
  // from_tab[(g * Q + q2) * L + l]: states of unit g reaching q2 on label l
  std::vector<uint32_t> ft((size_t)G * Q * L, 0);
  std::vector<QueryDesc> descs(G);
  std::vector<uint32_t> finals(G);
  for (uint32_t k = 0; k < G; k++) {
    const HostQuery &hq = query_host(units[k].q);
    descs[k] = hq.d;
    finals[k] = hq.d.final_mask;
    const uint32_t nl = hq.d.n_labels;
    for (uint32_t q = 0; q < hq.d.n_states; q++)
      for (uint32_t l = 0; l < std::min(nl, L); l++) {
        const int32_t q2 = hq.next[(size_t)q * nl + l];
        if (q2 >= 0) ft[((size_t)k * Q + q2) * L + l] |= 1u << q;
      }
  }
  // the union automaton: bottom-up iteration order and cost estimates
  QueryDesc un;
  std::memset(&un, 0, sizeof(un));
  un.n_states = Q;
  un.n_labels = L;
  uint32_t cnt = 0;
  for (uint32_t q2 = 0; q2 < Q; q2++) {
    un.in_begin[q2] = (uint16_t)cnt;
    for (uint32_t l = 0; l < L; l++) {
      uint32_t f = 0;
      for (uint32_t k = 0; k < G; k++) f |= ft[((size_t)k * Q + q2) * L + l];
      if (!f) continue;
      if (cnt >= RPQ_MAX_TRANSITIONS) return set_err(ctx, RPQ_ERR_TOO_COMPLEX, "union automaton too large");
      un.in_label[cnt] = (uint8_t)l;
      un.in_from[cnt] = f;
      cnt++;
    }
  }
  un.in_begin[Q] = (uint16_t)cnt;
  for (uint32_t k = 0; k < G; k++) un.final_mask |= finals[k];
  if (ctx->bpsm_multi == 0 && msbfs_multi_max_blocks(BFS_THREADS_HOST, &ctx->bpsm_multi))
    return set_err(ctx, RPQ_ERR_CUDA, "occupancy query failed");
  const int blocks = ctx_sm_share(ctx) * ctx->bpsm_multi;
  if (blocks <= 0) return set_err(ctx, RPQ_ERR_CUDA, "traversal kernel cannot be made resident");
  const uint64_t slack = 2ull * blocks * (BFS_THREADS_HOST / 32) * APPEND_SEG;
  const uint64_t words = (uint64_t)G * Q * n;
  {
    // traversal state grows with units x states x vertices: halve the launch
    // while it does not fit the budget
    const uint64_t need = workspace_bytes(words, words + slack, 0, G * 64);
    const uint64_t have = ctx->budget - ctx->used +
                          workspace_bytes(ctx->ws.vis_words, ctx->ws.list_cap, ctx->ws.claim_cap, ctx->ws.lane_cap);
    if (need + (64ull << 20) > have && G > 1) {
      const size_t h = G / 2;
      std::vector<MultiUnit> a(units.begin(), units.begin() + h), b(units.begin() + h, units.end());
      std::vector<uint64_t> la, lb;
      int r = rpq_lane_stats_multi(ctx, gr, a, &la, stats);
      if (r == RPQ_OK) r = rpq_lane_stats_multi(ctx, gr, b, &lb, stats);
      if (r) return r;
      std::copy(la.begin(), la.end(), lane_stats->begin());
      std::copy(lb.begin(), lb.end(), lane_stats->begin() + la.size());
      return RPQ_OK;
    }
  }
  int rc = ensure_workspace(ctx, words, words + slack, 0, G * 64);
  if (rc) return rc;
  Workspace &w = ctx->ws;
  // lanes: unit k's start vertices in lanes [64k, 64k + size); a unit with the
  // empty language keeps its lanes empty (it has no rows and no product vertices)
  std::vector<uint32_t> lanes((size_t)G * 64, NO_SOURCE);
  std::vector<uint64_t> empty(G, 0);
  for (uint32_t k = 0; k < G; k++) {
    const bool live = query_host(units[k].q).d.n_states > 0;
    for (uint32_t i = 0; i < 64; i++) {
      if (live && i < units[k].srcs.size()) {
        if (units[k].srcs[i] >= n) return set_err(ctx, RPQ_ERR_INVALID_ARG, "source id out of range");
        lanes[(size_t)k * 64 + i] = units[k].srcs[i];
      } else {
        empty[k] |= 1ull << i;
      }
    }
  }
  QueryDesc *d_desc = nullptr;
  u32 *d_ft = nullptr, *d_fin = nullptr;
  u64 *ls = nullptr;
  auto release = [&]() {
    dfree(ctx, d_desc, G);
    dfree(ctx, d_ft, ft.size());
    dfree(ctx, d_fin, G);
    dfree(ctx, ls, 3ull * G * 64);
  };
  if ((rc = dalloc(ctx, &d_desc, G)) || (rc = dalloc(ctx, &d_ft, ft.size())) || (rc = dalloc(ctx, &d_fin, G)) ||
      (rc = dalloc(ctx, &ls, 3ull * G * 64))) {
    release();
    return rc;
  }
  cudaStream_t st = ctx->stream;
  cudaError_t e = cudaMemcpyAsync(d_desc, descs.data(), G * sizeof(QueryDesc), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_ft, ft.data(), ft.size() * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_fin, finals.data(), G * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w.lanesrc, lanes.data(), lanes.size() * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w.empty, empty.data(), G * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ls, 0, 24ull * G * 64, st);
  if (e != cudaSuccess) {
    release();
    return cuda_err(ctx, e, "multi upload");
  }
  BfsParams p;
  std::memset(&p, 0, sizeof(p));
  p.out_off = g.out_off;
  p.out_col = g.out_col;
  p.in_off = g.in_off;
  p.in_col = g.in_col;
  p.hchunk = g.hchunk_in;
  for (uint32_t l = 0; l <= g.L && l < g.hchunk_in_off.size(); l++) p.hchunk_off[l] = g.hchunk_in_off[l];
  for (uint32_t l = 0; l < g.L; l++) p.label_edges[l] = g.label_edges[l];
  p.n = n;
  p.L = L;
  p.G = G;
  p.Q = Q;
  p.lanesrc = w.lanesrc;
  p.vis = w.vis;
  p.fr0 = w.fr0;
  p.fr1 = w.fr1;
  p.claim = nullptr;  // one word per group: claims come from the OR itself
  p.spill = w.spill;
  p.spill_cap = ctx->spill_cap;
  p.list0 = w.list0;
  p.list1 = w.list1;
  p.fbits = w.fbits;
  p.fbits_words = w.fbits_words();
  p.append_seg = APPEND_SEG;
  p.list_cap = w.list_cap;
  p.ctl = ctx->ctl;
  p.stamp_base = ctx->stamp;
  p.nblocks = (unsigned)blocks;
  p.force = 0;
  p.alpha = ctx->alpha;
  p.pull_dynamic = ctx->pull_dynamic;
  p.lane_by_source = ctx->lane_by_source;
  p.time_limit_ns = ctx->time_limit_ns;
  p.q = un;
  p.qg = d_desc;
  p.from_tab = d_ft;
  EmitParams ep{};
  ep.vis = w.vis;
  ep.n = n;
  ep.G = G;
  ep.Q = Q;
  ep.final_mask = un.final_mask;
  ep.final_g = d_fin;
  ep.lanesrc = w.lanesrc;
  ep.segs = (n + EMIT_SEG - 1) / EMIT_SEG;
  BfsCtl hctl;
  std::vector<uint64_t> hls(3ull * G * 64);
  if ((e = launch_vis_init(1, p, w.empty, st)) == cudaSuccess && (e = cudaMemsetAsync(ctx->ctl, 0, sizeof(BfsCtl), st)) == cudaSuccess &&
      (e = cudaEventRecord(ctx->ev[0], st)) == cudaSuccess && (e = launch_msbfs_multi(p, blocks, BFS_THREADS_HOST, st)) == cudaSuccess &&
      (e = cudaEventRecord(ctx->ev[1], st)) == cudaSuccess && (e = launch_emit_lane_stats(1, ep, ls, st)) == cudaSuccess &&
      (e = cudaEventRecord(ctx->ev[2], st)) == cudaSuccess)
    e = cudaMemcpyAsync(&hctl, ctx->ctl, sizeof(BfsCtl), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hls.data(), ls, hls.size() * 8, cudaMemcpyDeviceToHost, st);
  release();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_err(ctx, e, "multi-automaton launch");
  if (hctl.err) return traversal_error(ctx, hctl.err);
  ctx->stamp += (uint32_t)hctl.levels + 3;
  size_t at = 0;
  for (uint32_t k = 0; k < G; k++)
    for (size_t i = 0; i < units[k].srcs.size(); i++, at++)
      for (int c = 0; c < 3; c++) (*lane_stats)[3 * at + c] = hls[3 * ((size_t)k * 64 + i) + c];
  if (stats) {
    float ms_bfs = 0, ms_emit = 0;
    cudaEventElapsedTime(&ms_bfs, ctx->ev[0], ctx->ev[1]);
    cudaEventElapsedTime(&ms_emit, ctx->ev[1], ctx->ev[2]);
    stats->product_edges += hctl.stats[ST_W];
    stats->product_vertices += hctl.stats[ST_N];
    stats->levels += hctl.levels;
    stats->push_levels += hctl.stats[ST_PUSH_LEVELS];
    stats->pull_levels += hctl.stats[ST_PULL_LEVELS];
    stats->alg_bytes += hctl.stats[ST_ALG_BYTES];
    stats->group_product_edges += hctl.stats[ST_GROUP_W];
    stats->group_label_rows += hctl.stats[ST_GROUP_X];
    stats->bfs_ms += ms_bfs;
    stats->emit_ms += ms_emit;
    stats->bfs_launches += 1;
    stats->launches += 4;
  }
  return RPQ_OK;
}

// One lane-mode launch over tasks[idx[0 .. k)] (one lane each, lane i =
// idx[i]); results into lane_stats at the tasks' indices.
double host_seconds() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static int lane_launch(rpq_ctx *ctx, const rpq_graph *gr, const std::vector<LaneTask> &tasks, const uint32_t *idx,
                       uint32_t k, std::vector<uint64_t> *lane_stats, rpq_stats *stats, std::vector<double> *done_s) {
  const DevGraph &g = gr->g;
  const uint32_t n = g.n, L = g.L;
  const int nw = k <= 64 ? 1 : 4;
  const uint32_t K = 64u * nw;
  const uint32_t G = (k + K - 1) / K;
  if (G > 16) return set_err(ctx, RPQ_ERR_INVALID_ARG, "at most 4,096 lanes per lane-mode launch");
  const uint64_t GW = (uint64_t)G * nw;
  uint32_t Q = 0;
  for (uint32_t i = 0; i < k; i++) Q = std::max(Q, query_host(tasks[idx[i]].q).d.n_states);
  if (Q == 0) return RPQ_OK;
  // the union's transitions (state, label, target), in that order
  std::vector<uint8_t> used((size_t)Q * L * Q, 0);
  for (uint32_t i = 0; i < k; i++) {
    const HostQuery &hq = query_host(tasks[idx[i]].q);
    const uint32_t nl = hq.d.n_labels;
    for (uint32_t q = 0; q < hq.d.n_states; q++)
      for (uint32_t l = 0; l < std::min(nl, L); l++) {
        const int32_t t = hq.next[(size_t)q * nl + l];
        if (t >= 0) used[((size_t)q * L + l) * Q + t] = 1;
      }
  }
  std::vector<uint32_t> tid((size_t)Q * L * Q, 0xFFFFFFFFu);
  std::vector<uint16_t> out_begin(Q + 1, 0);
  std::vector<uint32_t> trans;
  for (uint32_t q = 0; q < Q; q++) {
    out_begin[q] = (uint16_t)trans.size();
    for (uint32_t l = 0; l < L; l++)
      for (uint32_t t = 0; t < Q; t++)
        if (used[((size_t)q * L + l) * Q + t]) {
          tid[((size_t)q * L + l) * Q + t] = (uint32_t)trans.size();
          trans.push_back(l | (t << 16));
        }
  }
  out_begin[Q] = (uint16_t)trans.size();
  if (trans.size() >= 0xFFFF) return set_err(ctx, RPQ_ERR_TOO_COMPLEX, "union automaton too large");
  const uint32_t T = (uint32_t)trans.size();
  // the union's bottom-up form: per target state, per label, its source states
  QueryDesc un;
  std::memset(&un, 0, sizeof(un));
  un.n_states = Q;
  un.n_labels = L;
  std::vector<uint16_t> in_t;
  uint32_t cnt = 0;
  for (uint32_t t2 = 0; t2 < Q; t2++) {
    un.in_begin[t2] = (uint16_t)cnt;
    for (uint32_t l = 0; l < L; l++) {
      uint32_t from = 0;
      for (uint32_t q = 0; q < Q; q++)
        if (used[((size_t)q * L + l) * Q + t2]) from |= 1u << q;
      if (!from) continue;
      if (cnt >= RPQ_MAX_TRANSITIONS) return set_err(ctx, RPQ_ERR_TOO_COMPLEX, "union automaton too large");
      un.in_label[cnt] = (uint8_t)l;
      un.in_from[cnt] = from;
      for (uint32_t q = 0; q < Q; q++)
        in_t.push_back((from >> q) & 1u ? (uint16_t)tid[((size_t)q * L + l) * Q + t2] : (uint16_t)0xFFFF);
      cnt++;
    }
  }
  un.in_begin[Q] = (uint16_t)cnt;
  if (in_t.empty()) in_t.push_back(0xFFFF);
  // per-lane masks: transitions taken, accepting states, states absent
  std::vector<u64> mask((size_t)std::max(1u, T) * GW, 0), fin((size_t)Q * GW, 0), empty_q((size_t)Q * GW, 0);
  std::vector<uint32_t> lanes((size_t)G * K, NO_SOURCE);
  for (uint32_t i = 0; i < G * K; i++) {
    const uint64_t word = i / 64, bit = 1ull << (i % 64);
    if (i >= k) {
      for (uint32_t q = 0; q < Q; q++) empty_q[q * GW + word] |= bit;
      continue;
    }
    const LaneTask &tk = tasks[idx[i]];
    const HostQuery &hq = query_host(tk.q);
    if (tk.source >= n) return set_err(ctx, RPQ_ERR_INVALID_ARG, "source id out of range");
    lanes[i] = hq.d.n_states ? tk.source : NO_SOURCE;
    const uint32_t nl = hq.d.n_labels;
    for (uint32_t q = 0; q < Q; q++) {
      if (q >= hq.d.n_states) {
        empty_q[q * GW + word] |= bit;
        continue;
      }
      if ((hq.d.final_mask >> q) & 1u) fin[q * GW + word] |= bit;
      for (uint32_t l = 0; l < std::min(nl, L); l++) {
        const int32_t t = hq.next[(size_t)q * nl + l];
        if (t >= 0) mask[(size_t)tid[((size_t)q * L + l) * Q + t] * GW + word] |= bit;
      }
    }
    if (!hq.d.n_states)
      for (uint32_t q = 0; q < Q; q++) empty_q[q * GW + word] |= bit;
    un.final_mask |= hq.d.final_mask;
  }
  un.final_mask &= Q >= 32 ? ~0u : ((1u << Q) - 1u);
  // resident blocks of the lane-mode kernel
  int &bpsm = ctx->bpsm_lane[nw == 1 ? 0 : 1];
  if (bpsm == 0 && msbfs_lane_max_blocks(nw, BFS_THREADS_HOST, &bpsm))
    return set_err(ctx, RPQ_ERR_CUDA, "occupancy query failed");
  const int blocks = ctx_sm_share(ctx) * bpsm;
  if (blocks <= 0) return set_err(ctx, RPQ_ERR_CUDA, "traversal kernel cannot be made resident");
  const uint64_t slack = 2ull * blocks * (BFS_THREADS_HOST / 32) * APPEND_SEG;
  const uint64_t words = (uint64_t)G * Q * n * nw;
  const uint64_t lists = (uint64_t)G * Q * n + slack;
  const uint64_t claims = nw > 1 ? (uint64_t)G * Q * n : 0;
  {
    const uint64_t need = workspace_bytes(words, lists, claims, G * K);
    const uint64_t have = ctx->budget - ctx->used +
                          workspace_bytes(ctx->ws.vis_words, ctx->ws.list_cap, ctx->ws.claim_cap, ctx->ws.lane_cap);
    if (need + (64ull << 20) > have) {
      if (k == 1) return set_err(ctx, RPQ_ERR_OUT_OF_BUDGET, "one lane's traversal state exceeds the budget");
      const uint32_t h = k / 2;
      int r = lane_launch(ctx, gr, tasks, idx, h, lane_stats, stats, done_s);
      if (r == RPQ_OK) r = lane_launch(ctx, gr, tasks, idx + h, k - h, lane_stats, stats, done_s);
      return r;
    }
  }
  int rc = ensure_workspace(ctx, words, lists, claims, G * K);
  if (rc) return rc;
  Workspace &w = ctx->ws;
  // the union's transitions grouped by (state, label) -- consecutive in
  // `trans` -- with the OR of each group's lane masks (the commit counts a
  // group's lanes with one mask)
  std::vector<uint16_t> grp_begin(Q + 1, 0);
  std::vector<uint32_t> grp;
  std::vector<u64> gmask;
  for (uint32_t q = 0; q < Q; q++) {
    grp_begin[q] = (uint16_t)grp.size();
    for (uint32_t t = out_begin[q]; t < out_begin[q + 1];) {
      const uint32_t l = trans[t] & 0xFFFFu;
      const size_t base = gmask.size();
      gmask.resize(base + GW, 0);
      uint32_t c = 0;
      for (; t < out_begin[q + 1] && (trans[t] & 0xFFFFu) == l; t++, c++)
        for (uint64_t k = 0; k < GW; k++) gmask[base + k] |= mask[(size_t)t * GW + k];
      grp.push_back(l | (c << 16));
    }
  }
  grp_begin[Q] = (uint16_t)grp.size();
  if (grp.empty()) {  // no transition: keep the buffers non-empty
    grp.push_back(0xFFFFu);
    gmask.assign(GW, 0);
  }
  // one upload buffer for the tables
  const size_t b_ob = (Q + 1) * 2, b_tr = std::max<size_t>(1, T) * 4, b_it = in_t.size() * 2;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t o_mask = 0, o_fin = o_mask + al(mask.size() * 8), o_emp = o_fin + al(fin.size() * 8),
               o_ob = o_emp + al(empty_q.size() * 8), o_tr = o_ob + al(b_ob), o_it = o_tr + al(b_tr),
               o_gm = o_it + al(b_it), o_gb = o_gm + al(gmask.size() * 8), o_gr = o_gb + al(grp_begin.size() * 2),
               o_ls = o_gr + al(grp.size() * 4), tbytes = o_ls + al(24ull * G * K);
  std::vector<unsigned char> host(o_ls);
  std::memcpy(host.data() + o_mask, mask.data(), mask.size() * 8);
  std::memcpy(host.data() + o_fin, fin.data(), fin.size() * 8);
  std::memcpy(host.data() + o_emp, empty_q.data(), empty_q.size() * 8);
  std::memcpy(host.data() + o_ob, out_begin.data(), b_ob);
  if (T) std::memcpy(host.data() + o_tr, trans.data(), b_tr);
  std::memcpy(host.data() + o_it, in_t.data(), b_it);
  std::memcpy(host.data() + o_gm, gmask.data(), gmask.size() * 8);
  std::memcpy(host.data() + o_gb, grp_begin.data(), grp_begin.size() * 2);
  std::memcpy(host.data() + o_gr, grp.data(), grp.size() * 4);
  unsigned char *dt = nullptr;
  if ((rc = dalloc(ctx, &dt, tbytes))) return rc;
  cudaStream_t st = ctx->stream;
  u64 *ls = reinterpret_cast<u64 *>(dt + o_ls);
  cudaError_t e = cudaMemcpyAsync(dt, host.data(), o_ls, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ls, 0, 24ull * G * K, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w.lanesrc, lanes.data(), lanes.size() * 4, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    dfree(ctx, dt, tbytes);
    return cuda_err(ctx, e, "lane tables upload");
  }
  BfsParams p;
  std::memset(&p, 0, sizeof(p));
  p.out_off = g.out_off;
  p.out_col = g.out_col;
  p.in_off = g.in_off;
  p.in_col = g.in_col;
  p.hchunk = g.hchunk_in;
  for (uint32_t l = 0; l <= g.L && l < g.hchunk_in_off.size(); l++) p.hchunk_off[l] = g.hchunk_in_off[l];
  for (uint32_t l = 0; l < g.L; l++) p.label_edges[l] = g.label_edges[l];
  p.n = n;
  p.L = L;
  p.G = G;
  p.Q = Q;
  p.lanesrc = w.lanesrc;
  p.vis = w.vis;
  p.fr0 = w.fr0;
  p.fr1 = w.fr1;
  p.claim = w.claim;
  p.spill = w.spill;
  p.spill_cap = ctx->spill_cap;
  p.list0 = w.list0;
  p.list1 = w.list1;
  p.fbits = w.fbits;
  p.fbits_words = w.fbits_words();
  p.append_seg = APPEND_SEG;
  p.list_cap = w.list_cap;
  p.ctl = ctx->ctl;
  p.stamp_base = ctx->stamp;
  p.nblocks = (unsigned)blocks;
  p.force = 0;
  p.alpha = ctx->alpha;
  p.pull_dynamic = ctx->pull_dynamic;
  p.lane_by_source = ctx->lane_by_source;
  p.time_limit_ns = ctx->time_limit_ns;
  p.q = un;
  p.alpha = ctx->lane_alpha;
  p.la_out_begin = reinterpret_cast<const unsigned short *>(dt + o_ob);
  p.la_trans = reinterpret_cast<const unsigned int *>(dt + o_tr);
  p.la_mask = reinterpret_cast<const unsigned long long *>(dt + o_mask);
  p.la_in_t = reinterpret_cast<const unsigned short *>(dt + o_it);
  p.la_grp_begin = reinterpret_cast<const unsigned short *>(dt + o_gb);
  p.la_grp = reinterpret_cast<const unsigned int *>(dt + o_gr);
  p.la_gmask = reinterpret_cast<const unsigned long long *>(dt + o_gm);
  EmitParams ep{};
  ep.vis = w.vis;
  ep.n = n;
  ep.G = G;
  ep.Q = Q;
  ep.final_mask = un.final_mask;
  ep.final_lane = reinterpret_cast<const unsigned long long *>(dt + o_fin);
  ep.lanesrc = w.lanesrc;
  ep.segs = (n + EMIT_SEG - 1) / EMIT_SEG;
  BfsCtl hctl;
  std::vector<uint64_t> hls(3ull * G * K);
  if ((e = launch_vis_init_lane(nw, p, reinterpret_cast<const u64 *>(dt + o_emp), st)) == cudaSuccess &&
      (e = cudaMemsetAsync(ctx->ctl, 0, sizeof(BfsCtl), st)) == cudaSuccess &&
      (e = cudaEventRecord(ctx->ev[0], st)) == cudaSuccess &&
      (e = launch_msbfs_lane(nw, p, blocks, BFS_THREADS_HOST, st)) == cudaSuccess &&
      (e = cudaEventRecord(ctx->ev[1], st)) == cudaSuccess && (e = launch_emit_lane_stats(nw, ep, ls, st)) == cudaSuccess &&
      (e = cudaEventRecord(ctx->ev[2], st)) == cudaSuccess)
    e = rb_queue(ctx, 0, ctx->ctl, sizeof(BfsCtl));
  if (e == cudaSuccess) e = cudaMemcpyAsync(hls.data(), ls, hls.size() * 8, cudaMemcpyDeviceToHost, st);
  dfree(ctx, dt, tbytes);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_err(ctx, e, "lane-mode launch");
  std::memcpy(&hctl, ctx->rb_host, sizeof(BfsCtl));
  if (hctl.err) return traversal_error(ctx, hctl.err);
  ctx->stamp += (uint32_t)hctl.levels + 3;
  const double now = host_seconds();
  for (uint32_t i = 0; i < k; i++) {
    for (int c = 0; c < 3; c++) (*lane_stats)[3ull * idx[i] + c] = hls[3ull * i + c];
    if (done_s) (*done_s)[idx[i]] = now;
  }
  if (ctx->trace) {
    uint32_t nl = (uint32_t)std::min<uint64_t>(hctl.levels, TRACE_LEVELS);
    std::fprintf(stderr, "[rpq trace] lanes k=%u G=%u NW=%d Q=%u T=%u levels=%llu W=%llu\n", k, G, nw, Q, T,
                 (unsigned long long)hctl.levels, (unsigned long long)hctl.stats[ST_W]);
    for (uint32_t l = 0; l < nl; l++)
      std::fprintf(stderr, "[rpq trace]   level %2u %s n=%10llu mf=%12llu %9.3f ms (commit %7.3f ms)\n", l,
                   hctl.trace_mode[l] == 1 ? "push" : "pull", (unsigned long long)hctl.trace_n[l],
                   (unsigned long long)hctl.trace_mf[l], (hctl.trace_t[l + 1] - hctl.trace_t[l]) * 1e-6,
                   hctl.trace_c[l] ? (hctl.trace_t[l + 1] - hctl.trace_c[l]) * 1e-6 : 0.0);
  }
  if (stats) {
    float ms_bfs = 0, ms_emit = 0;
    cudaEventElapsedTime(&ms_bfs, ctx->ev[0], ctx->ev[1]);
    cudaEventElapsedTime(&ms_emit, ctx->ev[1], ctx->ev[2]);
    stats->product_edges += hctl.stats[ST_W];
    stats->product_vertices += hctl.stats[ST_N];
    stats->levels += hctl.levels;
    stats->push_levels += hctl.stats[ST_PUSH_LEVELS];
    stats->pull_levels += hctl.stats[ST_PULL_LEVELS];
    stats->group_edges += hctl.stats[ST_GROUP_EDGES];
    stats->group_rows += hctl.stats[ST_GROUP_ROWS];
    stats->group_vertices += hctl.stats[ST_GROUP_VERTICES];
    stats->pull_edges += hctl.stats[ST_PULL_EDGES];
    stats->pull_vertices += hctl.stats[ST_PULL_VERTICES];
    stats->alg_bytes += hctl.stats[ST_ALG_BYTES];
    stats->group_product_edges += hctl.stats[ST_GROUP_W];
    stats->group_label_rows += hctl.stats[ST_GROUP_X];
    stats->lane_groups += G;
    stats->bfs_ms += ms_bfs;
    stats->emit_ms += ms_emit;
    stats->bfs_launches += 1;
    stats->launches += 6;
  }
  return RPQ_OK;
}

int rpq_lane_stats_lanes(rpq_ctx *ctx, const rpq_graph *gr, const std::vector<LaneTask> &tasks, uint32_t max_lanes,
                         std::vector<uint64_t> *lane_stats, rpq_stats *stats, std::vector<double> *done_s) {
  lane_stats->assign(3 * tasks.size(), 0);
  if (done_s) done_s->assign(tasks.size(), host_seconds());
  max_lanes = std::max(1u, std::min(max_lanes, 4096u));
  // tasks ordered by state count (a launch is sized by its largest automaton),
  // automata with more than 8 states apart from the rest
  std::vector<uint32_t> order;
  for (uint32_t i = 0; i < tasks.size(); i++) {
    if (!tasks[i].q) return set_err(ctx, RPQ_ERR_INVALID_ARG, "null query");
    if (query_host(tasks[i].q).d.n_states) order.push_back(i);
  }
  auto states = [&](uint32_t i) { return query_host(tasks[i].q).d.n_states; };
  std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return states(a) < states(b); });
  for (size_t b = 0; b < order.size();) {
    size_t e = std::min(order.size(), b + max_lanes);
    if (states(order[b]) <= 8)
      while (e > b + 1 && states(order[e - 1]) > 8) e--;
    const int rc = lane_launch(ctx, gr, tasks, order.data() + b, (uint32_t)(e - b), lane_stats, stats, done_s);
    if (rc) return rc;
    b = e;
  }
  return RPQ_OK;
}

void free_row_chunk(rpq_ctx *ctx, RowChunk &c) {
  dfree(ctx, c.lanesrc, c.n_lanes);
  dfree(ctx, c.lane_off, (uint64_t)c.n_lanes + 1);
  dfree(ctx, c.dst, c.rows);
  if (c.bits) {
    dfree(ctx, c.bits, (uint64_t)c.n_bits * c.bwords);
    dfree(ctx, c.lane_slot, c.n_lanes);
  }
  c = RowChunk{};
}

int make_tuple_result(rpq_ctx *ctx, uint32_t arity, u32 *tuples, uint64_t rows, uint64_t dsum, uint64_t dxor,
                      bool materialized, const rpq_stats &stats, rpq_result **out) {
  rpq_result *r = new rpq_result;
  r->ctx = ctx;
  ctx->live++;
  r->arity = arity;
  r->count = rows;
  r->dsum = dsum;
  r->dxor = dxor;
  r->materialized = materialized;
  r->tuples = tuples;
  r->tuple_bytes = tuples ? rows * arity * 4 : 0;
  r->stats = stats;
  *out = r;
  return RPQ_OK;
}

}  // namespace rpq
