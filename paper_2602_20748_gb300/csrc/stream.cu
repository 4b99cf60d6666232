// Streamed materialization: the sorted rows of one or more RPQs over a range
// of start vertices, delivered to the host one block at a time while the
// device keeps exploring (the batch-wise result transfer of the paper's
// Section 5, with a compact row layout).
//
// Two host threads drive the device:
//   * the evaluation thread runs the queries one after another, each over the
//     start vertices in batches of one traversal launch (eval + emission, the
//     rows stay on the device), and queues each finished batch; at most
//     MAX_PENDING batches wait to be copied, so the device memory held by rows
//     stays bounded;
//   * the copy thread splits a finished batch into pieces of at most SLOT_ROWS
//     destinations and copies each into a free pinned host slot on a copy
//     stream of its own, so the copy of batch k overlaps the traversal of
//     batch k + 1 on the context's stream.
// The caller takes filled slots in order through rpq_stream_next; a slot goes
// back to the copier when the caller asks for the next block.  Device memory
// of a copied batch is released by the evaluation thread (the only thread that
// allocates) once the copy's completion event has fired; the thread does not
// wait for copies in flight, so the next traversal starts while they run.
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "crpq.h"
#include "rpq_internal.h"

namespace {

constexpr uint64_t SLOT_ROWS = 1ull << 26;  // destinations per pinned slot (256 MiB)
constexpr int N_SLOTS = 3;
constexpr size_t MAX_PENDING = 2;  // evaluated batches not yet copied

// Pinned, device-mapped host buffer for a batch's lane metadata.
struct MetaBuf {
  void *h = nullptr;
  size_t bytes = 0;
};

struct Batch {
  uint32_t query = 0;  // index into the stream's queries
  std::vector<rpq::RowChunk> chunks;
  // host views of each chunk's lane sources and offsets, in `meta`: written
  // there by a kernel, so that they do not queue behind the bulk row copies
  // on the copy engine
  std::vector<const uint32_t *> lanesrc;
  std::vector<const uint64_t *> lane_off;
  MetaBuf meta;
  cudaEvent_t copied = nullptr;  // recorded after the batch's last copy
};

struct Slot {
  uint32_t *host = nullptr;  // pinned, SLOT_ROWS destinations
  cudaEvent_t done = nullptr;
  std::vector<uint32_t> sources;
  std::vector<uint64_t> offsets;
  uint64_t rows = 0;
  uint32_t query = 0;
};

}  // namespace

struct rpq_stream {
  rpq_ctx *ctx = nullptr;
  const rpq_graph *g = nullptr;
  std::vector<const rpq_query *> qs;
  uint32_t begin = 0, end = 0, batch = 4096;
  bool reverse = false;
  cudaStream_t copy = nullptr;
  Slot slots[N_SLOTS];
  std::mutex mu;
  std::condition_variable cv;
  std::deque<int> free_slots, ready;
  std::deque<Batch *> pending;  // evaluated, being or to be copied
  std::deque<Batch *> copied;   // copies issued; device rows to release
  std::vector<MetaBuf> meta_free;  // recycled metadata buffers
  int handed = -1;              // slot the caller holds
  bool eval_done = false, copy_done = false, stop = false;
  int rc = RPQ_OK;
  uint64_t rows = 0, dsum = 0, dxor = 0, blocks = 0;
  rpq_stats stats;
  std::thread t_eval, t_copy;
};

namespace {

// Lane metadata of the chunks [lanesrc | lane_off]: copied from the device
// into mapped pinned memory by this kernel (one word per thread).
__global__ void meta_to_host(const uint32_t *__restrict__ lanesrc, const unsigned long long *__restrict__ lane_off,
                             uint32_t n_lanes, uint32_t *h_lanesrc, unsigned long long *h_lane_off) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= n_lanes; i += gridDim.x * blockDim.x) {
    if (i < n_lanes) h_lanesrc[i] = lanesrc[i];
    h_lane_off[i] = lane_off[i];
  }
}

int meta_get(rpq_stream *s, size_t bytes, MetaBuf *out) {
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (size_t i = 0; i < s->meta_free.size(); i++)
      if (s->meta_free[i].bytes >= bytes) {
        *out = s->meta_free[i];
        s->meta_free.erase(s->meta_free.begin() + i);
        return RPQ_OK;
      }
  }
  const size_t want = (bytes + 65535) & ~(size_t)65535;
  cudaError_t e = cudaHostAlloc(&out->h, want, cudaHostAllocMapped);
  if (e != cudaSuccess) {
    out->h = nullptr;
    return rpq::ctx_error(s->ctx, RPQ_ERR_CUDA, std::string("stream metadata buffer: ") + cudaGetErrorString(e));
  }
  out->bytes = want;
  return RPQ_OK;
}

void meta_put(rpq_stream *s, MetaBuf m) {
  if (!m.h) return;
  std::lock_guard<std::mutex> lk(s->mu);
  s->meta_free.push_back(m);
}

void release_batch(rpq_stream *s, Batch *b) {
  if (b->copied) {
    cudaEventSynchronize(b->copied);
    cudaEventDestroy(b->copied);
  }
  for (rpq::RowChunk &c : b->chunks) rpq::free_row_chunk(s->ctx, c);
  meta_put(s, b->meta);
  delete b;
}

// Brings the lane sources and offsets of b's chunks to the host (see Batch).
int fetch_meta(rpq_stream *s, Batch *b) {
  size_t bytes = 0;
  for (const rpq::RowChunk &c : b->chunks) bytes += ((size_t)c.n_lanes + 1) * 8 + (size_t)c.n_lanes * 4 + 8;
  if (bytes == 0) return RPQ_OK;
  int rc = meta_get(s, bytes, &b->meta);
  if (rc != RPQ_OK) return rc;
  cudaStream_t cs = rpq::ctx_stream(s->ctx);
  char *h = static_cast<char *>(b->meta.h);
  cudaError_t e = cudaSuccess;
  for (const rpq::RowChunk &c : b->chunks) {
    auto *h_off = reinterpret_cast<uint64_t *>(h);  // 8-byte aligned: each chunk's part is rounded up to 8
    auto *h_src = reinterpret_cast<uint32_t *>(h + ((size_t)c.n_lanes + 1) * 8);
    void *d_off = nullptr, *d_src = nullptr;
    if ((e = cudaHostGetDevicePointer(&d_off, h_off, 0)) != cudaSuccess ||
        (e = cudaHostGetDevicePointer(&d_src, h_src, 0)) != cudaSuccess)
      break;
    meta_to_host<<<(c.n_lanes + 256) / 256, 256, 0, cs>>>(c.lanesrc, c.lane_off, c.n_lanes,
                                                          static_cast<uint32_t *>(d_src),
                                                          static_cast<unsigned long long *>(d_off));
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    b->lane_off.push_back(h_off);
    b->lanesrc.push_back(h_src);
    h += (((size_t)c.n_lanes + 1) * 8 + (size_t)c.n_lanes * 4 + 7) & ~(size_t)7;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e != cudaSuccess) return rpq::ctx_error(s->ctx, RPQ_ERR_CUDA, std::string("stream: ") + cudaGetErrorString(e));
  return RPQ_OK;
}

// Releases the copied batches whose copies have completed (all of them when
// wait is set); the others stay queued.
void release_copied(rpq_stream *s, bool wait) {
  std::vector<Batch *> done;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto it = s->copied.begin(); it != s->copied.end();) {
      if (wait || !(*it)->copied || cudaEventQuery((*it)->copied) != cudaErrorNotReady) {
        done.push_back(*it);
        it = s->copied.erase(it);
      } else {
        ++it;
      }
    }
  }
  for (Batch *b : done) release_batch(s, b);
}

void eval_thread(rpq_stream *s) {
  cudaSetDevice(rpq::ctx_device(s->ctx));
  bool failed = false;
  for (uint32_t qi = 0; qi < s->qs.size() && !failed; qi++) {
    for (uint64_t b0 = s->begin; b0 < s->end; b0 += s->batch) {
      release_copied(s, false);
      {
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv.wait(lk, [&] { return s->stop || s->pending.size() < MAX_PENDING; });
        if (s->stop) {
          failed = true;
          break;
        }
      }
      const uint32_t e = (uint32_t)std::min<uint64_t>(s->end, b0 + s->batch);
      std::vector<uint32_t> srcs(e - (uint32_t)b0);
      for (uint32_t i = 0; i < srcs.size(); i++) srcs[i] = (uint32_t)b0 + i;
      auto *b = new Batch;
      b->query = qi;
      rpq_stats st;
      std::memset(&st, 0, sizeof(st));
      uint64_t hs = 0, hx = 0;
      int rc = rpq::rpq_rows_for_sources(s->ctx, s->g, s->qs[qi], srcs, s->reverse, &b->chunks, &st, &hs, &hx);
      uint64_t nrows = 0;
      if (rc == RPQ_OK) rc = fetch_meta(s, b);
      if (rc == RPQ_OK)
        for (const rpq::RowChunk &c : b->chunks) nrows += c.rows;
      std::lock_guard<std::mutex> lk(s->mu);
      if (rc != RPQ_OK) {
        s->rc = rc;
        s->copied.push_back(b);  // released below
        failed = true;
        break;
      }
      s->rows += nrows;
      s->dsum += hs;
      s->dxor ^= hx;
      rpq_stats &a = s->stats;
      a.product_edges += st.product_edges;
      a.product_vertices += st.product_vertices;
      a.levels += st.levels;
      a.push_levels += st.push_levels;
      a.pull_levels += st.pull_levels;
      a.group_edges += st.group_edges;
      a.group_rows += st.group_rows;
      a.group_vertices += st.group_vertices;
      a.pull_edges += st.pull_edges;
      a.pull_vertices += st.pull_vertices;
      a.lane_words = st.lane_words ? st.lane_words : a.lane_words;
      a.lane_groups += st.lane_groups;
      a.bfs_ms += st.bfs_ms;
      a.emit_ms += st.emit_ms;
      a.bfs_launches += st.bfs_launches;
      a.launches += st.launches;
      a.alg_bytes += st.alg_bytes;
      a.group_product_edges += st.group_product_edges;
      a.group_label_rows += st.group_label_rows;
      s->pending.push_back(b);
      s->cv.notify_all();
    }
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->eval_done = true;
  s->cv.notify_all();
}

void copy_thread(rpq_stream *s) {
  cudaSetDevice(rpq::ctx_device(s->ctx));
  for (;;) {
    Batch *b = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait(lk, [&] { return s->stop || !s->pending.empty() || s->eval_done; });
      if (s->stop || s->pending.empty()) {
        s->copy_done = true;
        s->cv.notify_all();
        return;
      }
      b = s->pending.front();
    }
    bool ok = true;
    for (size_t ci = 0; ci < b->chunks.size() && ok; ci++) {
      const rpq::RowChunk &c = b->chunks[ci];
      const uint64_t *off = b->lane_off[ci];
      const uint32_t *lsrc = b->lanesrc[ci];
      uint32_t lane = 0;
      for (uint64_t r0 = 0; r0 < c.rows && ok;) {
        int si;
        {
          std::unique_lock<std::mutex> lk(s->mu);
          s->cv.wait(lk, [&] { return s->stop || !s->free_slots.empty(); });
          if (s->stop) {
            ok = false;
            break;
          }
          si = s->free_slots.front();
          s->free_slots.pop_front();
        }
        Slot &sl = s->slots[si];
        const uint64_t k = std::min<uint64_t>(SLOT_ROWS, c.rows - r0);
        cudaError_t ce = cudaMemcpyAsync(sl.host, c.dst + r0, k * 4, cudaMemcpyDeviceToHost, s->copy);
        if (ce == cudaSuccess) ce = cudaEventRecord(sl.done, s->copy);
        // lanes whose rows meet [r0, r0 + k), with offsets relative to r0
        sl.sources.clear();
        sl.offsets.clear();
        while (lane < c.n_lanes && off[lane + 1] <= r0) lane++;
        for (uint32_t i = lane; i < c.n_lanes && off[i] < r0 + k; i++) {
          if (off[i + 1] <= off[i]) continue;  // no rows
          sl.sources.push_back(lsrc[i]);
          sl.offsets.push_back(std::max(off[i], r0) - r0);
        }
        sl.offsets.push_back(k);
        sl.rows = k;
        sl.query = b->query;
        std::lock_guard<std::mutex> lk(s->mu);
        if (ce != cudaSuccess) {
          s->rc = rpq::ctx_error(s->ctx, RPQ_ERR_CUDA, std::string("stream copy: ") + cudaGetErrorString(ce));
          s->free_slots.push_back(si);
          ok = false;
          break;
        }
        s->ready.push_back(si);
        s->blocks++;
        s->cv.notify_all();
        r0 += k;
      }
    }
    cudaEventCreateWithFlags(&b->copied, cudaEventDisableTiming);
    cudaEventRecord(b->copied, s->copy);
    std::lock_guard<std::mutex> lk(s->mu);
    s->pending.pop_front();
    s->copied.push_back(b);
    s->cv.notify_all();
    if (!ok) {
      s->copy_done = true;
      return;
    }
  }
}

void destroy_stream(rpq_stream *s) {
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->t_eval.joinable()) s->t_eval.join();
  if (s->t_copy.joinable()) s->t_copy.join();
  cudaSetDevice(rpq::ctx_device(s->ctx));
  if (s->copy) cudaStreamSynchronize(s->copy);
  for (Batch *b : s->pending) release_batch(s, b);
  for (Batch *b : s->copied) release_batch(s, b);
  for (MetaBuf &m : s->meta_free) cudaFreeHost(m.h);
  for (Slot &sl : s->slots)
    if (sl.done) cudaEventDestroy(sl.done);  // the pinned slots stay with the context
  if (s->copy) cudaStreamDestroy(s->copy);
  delete s;
}

}  // namespace

extern "C" {

int rpq_stream_open_multi(rpq_ctx *ctx, const rpq_graph *g, const rpq_query *const *queries, uint32_t n_queries,
                          uint32_t src_begin, uint32_t src_end, uint32_t flags, rpq_stream **out) {
  if (!ctx || !g || !queries || !out) return rpq::ctx_error(ctx, RPQ_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (n_queries == 0) return rpq::ctx_error(ctx, RPQ_ERR_INVALID_ARG, "no queries");
  for (uint32_t i = 0; i < n_queries; i++)
    if (!queries[i]) return rpq::ctx_error(ctx, RPQ_ERR_INVALID_ARG, "null query");
  const int dev = rpq::ctx_device(ctx);
  if (dev < 0) return rpq::ctx_error(ctx, RPQ_ERR_NO_DEVICE, "host-only context has no GPU");
  if (flags & ~(uint32_t)RPQ_REVERSE) return rpq::ctx_error(ctx, RPQ_ERR_INVALID_ARG, "flags: only RPQ_REVERSE");
  if (src_begin > src_end || src_end > rpq::graph_dev(g).n)
    return rpq::ctx_error(ctx, RPQ_ERR_INVALID_ARG, "bad source range");
  if (flags & RPQ_REVERSE)
    for (uint32_t i = 0; i < n_queries; i++)
      if (!rpq::query_host(queries[i]).has_rev)
        return rpq::ctx_error(ctx, RPQ_ERR_TOO_COMPLEX,
                              "the reversed language needs more than RPQ_MAX_STATES states");
  cudaSetDevice(dev);
  auto *s = new rpq_stream;
  s->ctx = ctx;
  s->g = g;
  s->qs.assign(queries, queries + n_queries);
  s->begin = src_begin;
  s->end = src_end;
  s->reverse = (flags & RPQ_REVERSE) != 0;
  s->batch = 64u * 4u * 16u;  // one traversal launch of 16 lane groups
  std::memset(&s->stats, 0, sizeof(s->stats));
  void *hosts[N_SLOTS];
  int prc = rpq::ctx_pinned(ctx, N_SLOTS, SLOT_ROWS * 4, hosts);
  cudaError_t e = cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking);
  for (int i = 0; i < N_SLOTS && e == cudaSuccess && prc == RPQ_OK; i++) {
    s->slots[i].host = (uint32_t *)hosts[i];
    e = cudaEventCreateWithFlags(&s->slots[i].done, cudaEventDisableTiming);
    s->free_slots.push_back(i);
  }
  if (e != cudaSuccess || prc != RPQ_OK) {
    s->eval_done = s->copy_done = true;
    std::string msg = prc != RPQ_OK ? std::string(rpq_last_error(ctx))
                                    : std::string("stream setup: ") + cudaGetErrorString(e);
    destroy_stream(s);
    return rpq::ctx_error(ctx, prc != RPQ_OK ? prc : RPQ_ERR_CUDA, msg);
  }
  s->t_eval = std::thread(eval_thread, s);
  s->t_copy = std::thread(copy_thread, s);
  *out = s;
  return RPQ_OK;
}

int rpq_stream_open(rpq_ctx *ctx, const rpq_graph *g, const rpq_query *q, uint32_t src_begin, uint32_t src_end,
                    uint32_t flags, rpq_stream **out) {
  if (!q) {
    if (out) *out = nullptr;
    return rpq::ctx_error(ctx, RPQ_ERR_INVALID_ARG, "null argument");
  }
  return rpq_stream_open_multi(ctx, g, &q, 1, src_begin, src_end, flags, out);
}

int rpq_stream_next(rpq_stream *s, rpq_row_block *block) {
  if (!s || !block) return RPQ_ERR_INVALID_ARG;
  std::memset(block, 0, sizeof(*block));
  int si;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->handed >= 0) {
      s->free_slots.push_back(s->handed);
      s->handed = -1;
      s->cv.notify_all();
    }
    s->cv.wait(lk, [&] { return !s->ready.empty() || s->copy_done; });
    if (s->ready.empty()) return s->rc;  // the end (or the error that ended it)
    si = s->ready.front();
    s->ready.pop_front();
    s->handed = si;
  }
  Slot &sl = s->slots[si];
  cudaError_t e = cudaEventSynchronize(sl.done);
  if (e != cudaSuccess) return rpq::ctx_error(s->ctx, RPQ_ERR_CUDA, std::string("stream: ") + cudaGetErrorString(e));
  block->n_sources = (uint32_t)sl.sources.size();
  block->sources = sl.sources.data();
  block->offsets = sl.offsets.data();
  block->dst = sl.host;
  block->n_rows = sl.rows;
  block->query = sl.query;
  return RPQ_OK;
}

int rpq_stream_info(rpq_stream *s, uint64_t *rows, uint64_t *digest_sum, uint64_t *digest_xor, rpq_stats *stats) {
  if (!s) return RPQ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (rows) *rows = s->rows;
  if (digest_sum) *digest_sum = s->dsum;
  if (digest_xor) *digest_xor = s->dxor;
  if (stats) *stats = s->stats;
  return RPQ_OK;
}

void rpq_stream_close(rpq_stream *s) {
  if (s) destroy_stream(s);
}

}  // extern "C"
