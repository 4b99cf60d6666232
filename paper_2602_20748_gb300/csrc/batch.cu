// Many single-source RPQs with different expressions in one persistent
// launch (the batched form of Definition 1 with one start vertex per query).
//
// The paper evaluates each traversal group in a thread block and notes that
// with few start vertices the GPU is poorly used (small-batch experiments,
// Section 7.3).  Here every query keeps a dense visited bitmap over its own
// (DFA state, vertex) pairs -- one bit each, Q_i * |V| bits -- and all
// queries advance together, level by level, in one cooperative kernel over a
// shared frontier list of (query, state, vertex) entries.  A level is
// expanded top-down: a warp takes 32 entries, spreads the out-edges of their
// transition rows evenly over its lanes, and test-and-sets the target bits
// (a plain read first, the atomic only when the bit is clear); rows longer
// than SPILL_EDGES are cut into chunks shared by all warps.  Results are the
// accepting states' bitmaps, emitted as (query index, vertex) rows.
#include <algorithm>
#include <atomic>
#include <thread>
#include <map>
#include <string>
#include <cstdio>
#include <cstring>
#include <vector>

#include "batch.h"
#include "crpq.h"
#include "device_common.cuh"
#include "rpq_internal.h"

namespace rpq {

namespace {

constexpr int BATCH_THREADS = 256;  // default block size (the autotuner may pick another)
constexpr int BATCH_MAX_THREADS = 512;
constexpr unsigned ERR_LIST_FULL = 100;  // frontier list capacity exceeded
// Bounds checks: an index outside its array records which check failed (the
// access is skipped) and stops the search with RPQ_ERR_CUDA on the host.
constexpr unsigned ERR_BOUNDS = 200;
// at most this many helper contexts evaluate evicted queries side by side
constexpr uint32_t MAX_REGROUP_STREAMS = 16;

struct BatchParams {
  const uint32_t *out_off;
  const uint32_t *out_col;
  uint32_t n;
  uint32_t L;
  uint32_t nq;
  const QueryDesc *qd;
  const u64 *vis_off;  // first word of query i's bitmaps
  const u32 *srcs;
  u64 *vis;
  u64 vis_words;       // size of vis
  u64 m;               // edges (size of out_col)
  u64 wps;             // words per state bitmap
  u64 *list0, *list1;
  u64 list_cap;
  u64 *spill;
  u64 spill_cap;       // spill records available (<= SPILL_CAP)
  BfsCtl *ctl;
  unsigned nblocks;
  u64 time_limit_ns;
  // per-query accounting and eviction (qn/qw may be null: no eviction)
  unsigned long long *qn;  // product vertices found per query
  unsigned long long *qw;  // product edges per query (W)
  u32 *evicted;            // 1 = query left the batch (too large)
  u64 evict_at;            // evict a query once qn exceeds this (0: never)
  u32 append_seg;          // list slots a warp reserves at a time (0: one atomic per append)
};

__device__ __forceinline__ u64 bentry(u32 i, u32 q, u32 v) { return ((u64)i << 37) | ((u64)q << 32) | v; }

__device__ __forceinline__ bool bad(const BatchParams &p, bool cond, unsigned which) {
  if (cond) atomicCAS(&p.ctl->err, 0u, ERR_BOUNDS + which);
  return cond;
}


// Reserves up to `chunks` spill records with one atomic add and returns how
// many of them fit below `cap` (their first index in *at).  Records below
// the capacity are always written by their reserver, so the spill phase,
// which reads min(count, cap) records, never reads one nobody wrote; the
// chunks that do not fit are processed in place.
__device__ __forceinline__ unsigned spill_reserve(unsigned long long *count, unsigned chunks, unsigned long long cap,
                                                  unsigned long long *at) {
  const unsigned long long first = atomicAdd(count, (unsigned long long)chunks);
  *at = first;
  if (first >= cap) return 0;
  return (unsigned)min((unsigned long long)chunks, cap - first);
}

__device__ bool bbarrier(BfsCtl *c, unsigned nblocks, u64 limit_ns) {
  __shared__ unsigned stop;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *gen = &c->bar_gen;
    unsigned g0 = *gen;
    __threadfence();
    unsigned arrived = atomicAdd(&c->bar_count, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(&c->bar_count, 0u);
      __threadfence();
      atomicAdd(&c->bar_gen, 1u);
    } else {
      u64 t0 = globaltimer_ns();
      unsigned spins = 0;
      while (*gen == g0) {
        __nanosleep(100);
        if ((++spins & 63u) == 0 && globaltimer_ns() - t0 > limit_ns) {
          atomicCAS(&c->err, 0u, (unsigned)(-RPQ_ERR_TIMEOUT));
          break;
        }
        if (*(volatile unsigned *)&c->err) break;
      }
    }
    __threadfence();
    stop = *(volatile unsigned *)&c->err;
  }
  __syncthreads();
  return stop == 0;
}

__device__ __forceinline__ u32 bdegsum(const BatchParams &p, const QueryDesc &qd, u32 q, u32 v) {
  u32 s = 0;
  for (u32 t = qd.out_begin[q]; t < qd.out_begin[q + 1]; t++) {
    u32 l = qd.out_label[t];
    if (l >= p.L || bad(p, v >= p.n, 4)) continue;
    const u32 *off = p.out_off + (u64)l * (p.n + 1) + v;
    s += __ldg(off + 1) - __ldg(off);
  }
  return s;
}

// A warp's current run of reserved list slots [pos, end) (warp-uniform).
struct BAppender {
  u64 pos = 0, end = 0;
};

// Warp-aggregated append with a capacity check; a full list stops the search
// with an error the host answers by splitting the batch.  The warp reserves
// append_seg slots at a time with one atomic add (the list counter would
// otherwise take one atomic per append from every warp); slots it does not
// use hold NO_ENTRY (bappend_close).  Small lists use one atomic per append.
__device__ __forceinline__ void bappend(const BatchParams &p, BAppender &a, bool take, u64 entry,
                                        unsigned long long *count, u64 *list) {
  const u32 b = __ballot_sync(FULL_MASK, take);
  if (!b) return;
  const u32 k = __popc(b), r = __popc(b & lanemask_lt());
  u64 at;
  if (p.append_seg == 0) {
    u64 base = 0;
    if (lane_id() == __ffs(b) - 1) base = atomicAdd(count, (unsigned long long)k);
    at = __shfl_sync(FULL_MASK, base, __ffs(b) - 1) + r;
  } else {
    const u64 room = a.end - a.pos;
    u64 nb = 0;
    if (k > room) {
      if (lane_id() == 0) nb = atomicAdd(count, (unsigned long long)p.append_seg);
      nb = __shfl_sync(FULL_MASK, nb, 0);
    }
    at = r < room ? a.pos + r : nb + (r - room);
    if (k > room) {
      a.pos = nb + (k - room);
      a.end = nb + p.append_seg;
    } else {
      a.pos += k;
    }
  }
  if (take) {
    if (at < p.list_cap)
      list[at] = entry;
    else
      atomicCAS(&p.ctl->err, 0u, ERR_LIST_FULL);
  }
}

__device__ __forceinline__ void bappend_close(const BatchParams &p, BAppender &a, u64 *list) {
  for (u64 i = a.pos + lane_id(); i < a.end; i += 32)
    if (i < p.list_cap) list[i] = NO_ENTRY;
  a.pos = a.end = 0;
}

// Test-and-set of (query i, state q2, vertex w); true when this thread set it.
__device__ __forceinline__ bool bvisit(const BatchParams &p, u32 i, u32 q2, u32 w) {
  if (bad(p, i >= p.nq, 1) || bad(p, w >= p.n, 2)) return false;
  const u64 at = p.vis_off[i] + (u64)q2 * p.wps + (w >> 6);
  if (bad(p, at >= p.vis_words || q2 >= p.qd[i].n_states, 3)) return false;
  u64 *word = p.vis + at;
  const u64 bit = 1ull << (w & 63);
  if (__ldcg(word) & bit) return false;
  return !(atomicOr((unsigned long long *)word, bit) & bit);
}

__device__ void bseed(const BatchParams &p, u64 *W, u64 *N) {
  const u64 stride = (u64)gridDim.x * blockDim.x;
  BAppender app;
  for (u64 base = (u64)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < p.nq; base += stride) {
    u64 i = base + lane_id();
    bool take = false;
    u32 s = 0;
    if (i < p.nq && p.qd[i].n_states > 0) {
      s = p.srcs[i];
      take = bvisit(p, (u32)i, 0, s);
      if (take) {
        const u32 d = bdegsum(p, p.qd[i], 0, s);
        *W += d;
        *N += 1;
        if (p.qn) {
          p.qn[i] = 1;
          p.qw[i] = d;
        }
      }
    }
    bappend(p, app, take, bentry((u32)i, 0, s), &p.ctl->n_list[0], p.list0);
  }
  bappend_close(p, app, p.list0);
}

__device__ void bpush(const BatchParams &p, int lp, u32 cur, u32 nxt, u64 n_cur, u64 *edges) {
  const u64 *list = lp ? p.list1 : p.list0;
  u64 *nlist = lp ? p.list0 : p.list1;
  const u32 lane = lane_id();
  BAppender app;
  for (;;) {
    u64 base = 0;
    if (lane == 0) base = atomicAdd(&p.ctl->cursor[cur], 32ull);
    base = __shfl_sync(FULL_MASK, base, 0);
    if (base >= n_cur) break;
    const u64 idx = base + lane;
    u64 e = idx < n_cur ? __ldcg(&list[idx]) : NO_ENTRY;
    const bool present = e != NO_ENTRY;
    if (!present) e = 0;
    const u32 i = (u32)(e >> 37), q = (u32)(e >> 32) & 31u, v = (u32)e;
    bool valid = present && !bad(p, i >= p.nq || v >= p.n, 10);
    if (valid && p.evict_at && __ldcg(&p.evicted[i])) valid = false;
    const QueryDesc *qd = p.qd + (valid ? i : 0);
    const u32 t_beg = valid ? qd->out_begin[q] : 0;
    const u32 nt = valid ? qd->out_begin[q + 1] - t_beg : 0;
    const u32 max_nt = __reduce_max_sync(FULL_MASK, nt);
    for (u32 j = 0; j < max_nt; j++) {
      u32 rbeg = 0, rlen = 0, q2 = 0;
      if (j < nt) {
        const u32 t = t_beg + j;
        const u32 l = qd->out_label[t];
        q2 = qd->out_to[t];
        if (l < p.L && !bad(p, v >= p.n || i >= p.nq, 5)) {
          const u32 *off = p.out_off + (u64)l * (p.n + 1) + v;
          rbeg = __ldg(off);
          rlen = __ldg(off + 1) - rbeg;
          if (bad(p, (u64)rbeg + rlen > p.m, 6)) rlen = 0;
        }
      }
      if (rlen > SPILL_EDGES) {
        const u32 chunks = (rlen + SPILL_EDGES - 1) / SPILL_EDGES;
        u64 at = 0;
        const u32 fit = spill_reserve(&p.ctl->spill_count[cur], chunks, p.spill_cap, &at);
        for (u32 c = 0; c < fit; c++) {
          u64 *rec = p.spill + (at + c) * 2;
          rec[0] = bentry(i, q2, 0) | (rbeg + c * SPILL_EDGES);
          rec[1] = min(SPILL_EDGES, rlen - c * SPILL_EDGES);
        }
        // the chunks that did not fit stay with this warp
        const u32 moved = min(rlen, fit * SPILL_EDGES);
        rbeg += moved;
        rlen -= moved;
      }
      u32 pre = rlen;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        u32 t = __shfl_up_sync(FULL_MASK, pre, o);
        if (lane >= (u32)o) pre += t;
      }
      const u32 total = __shfl_sync(FULL_MASK, pre, 31);
      pre -= rlen;
      *edges += (lane == 0) ? total : 0;
      for (u32 k0 = 0; k0 < total; k0 += 32) {
        const u32 k = k0 + lane;
        u32 o = 0;
#pragma unroll
        for (u32 step = 16; step > 0; step >>= 1) {
          u32 pv = __shfl_sync(FULL_MASK, pre, o + step);
          if (pv <= k) o += step;
        }
        const u32 o_beg = __shfl_sync(FULL_MASK, rbeg, o);
        const u32 o_pre = __shfl_sync(FULL_MASK, pre, o);
        const u32 o_q2 = __shfl_sync(FULL_MASK, q2, o);
        const u32 o_i = __shfl_sync(FULL_MASK, i, o);
        bool take = false;
        u32 w = 0;
        if (k < total && !bad(p, (u64)o_beg + (k - o_pre) >= p.m, 7)) {
          w = __ldg(p.out_col + o_beg + (k - o_pre));
          take = bvisit(p, o_i, o_q2, w);
        }
        bappend(p, app, take, bentry(o_i, o_q2, w), &p.ctl->n_list[nxt], nlist);
      }
    }
  }
  bappend_close(p, app, nlist);
}

__device__ void bspill(const BatchParams &p, int lp, u32 cur, u32 nxt, u64 *edges) {
  u64 *nlist = lp ? p.list0 : p.list1;
  const u32 lane = lane_id();
  const u64 count = min(*(volatile unsigned long long *)&p.ctl->spill_count[cur], (unsigned long long)p.spill_cap);
  BAppender app;
  for (;;) {
    u64 r = 0;
    if (lane == 0) r = atomicAdd(&p.ctl->spill_cursor[cur], 1ull);
    r = __shfl_sync(FULL_MASK, r, 0);
    if (r >= count) break;
    const u64 h = __ldcg(p.spill + 2 * r);
    const u32 len = (u32)__ldcg(p.spill + 2 * r + 1);
    const u32 i = (u32)(h >> 37), q2 = (u32)(h >> 32) & 31u, b = (u32)h;
    if (p.evict_at && i < p.nq && __ldcg(&p.evicted[i])) continue;  // warp-uniform
    *edges += (lane == 0) ? len : 0;
    for (u32 k0 = 0; k0 < len; k0 += 32) {
      const u32 k = k0 + lane;
      bool take = false;
      u32 w = 0;
      if (k < len && !bad(p, (u64)b + k >= p.m, 8)) {
        w = __ldg(p.out_col + b + k);
        take = bvisit(p, i, q2, w);
      }
      bappend(p, app, take, bentry(i, q2, w), &p.ctl->n_list[nxt], nlist);
    }
  }
  bappend_close(p, app, nlist);
}

__device__ void bcommit(const BatchParams &p, int lp, u32 nxt, u64 *W, u64 *N) {
  const u64 *nlist = lp ? p.list0 : p.list1;
  u64 n_next = *(volatile unsigned long long *)&p.ctl->n_list[nxt];
  if (n_next > p.list_cap) n_next = p.list_cap;
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 j0 = (u64)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); j0 < n_next; j0 += stride) {
    const u64 j = j0 + lane_id();
    bool ok = j < n_next;
    u32 i = 0;
    u64 d = 0;
    if (ok) {
      const u64 e = __ldcg(&nlist[j]);
      ok = e != NO_ENTRY;
    }
    if (ok) {
      const u64 e = __ldcg(&nlist[j]);
      i = (u32)(e >> 37);
      const u32 q = (u32)(e >> 32) & 31u, v = (u32)e;
      ok = !bad(p, i >= p.nq, 9);
      if (ok) d = bdegsum(p, p.qd[i], q, v);
    }
    *W += d;
    *N += ok ? 1 : 0;
    if (p.qn) {
      // per-query counters; the entries of a warp usually share one query
      const u32 i0 = __shfl_sync(FULL_MASK, i, 0);
      const bool same = __all_sync(FULL_MASK, !ok || i == i0);
      if (same) {
        const u64 dn = warp_sum((u64)(ok ? 1 : 0)), dw = warp_sum(d);
        if (lane_id() == 0 && dn) {
          const u64 before = atomicAdd(&p.qn[i0], dn);
          atomicAdd(&p.qw[i0], dw);
          if (p.evict_at && before + dn > p.evict_at) p.evicted[i0] = 1u;
        }
      } else if (ok) {
        const u64 before = atomicAdd(&p.qn[i], 1ull);
        atomicAdd(&p.qw[i], d);
        if (p.evict_at && before + 1 > p.evict_at) p.evicted[i] = 1u;
      }
    }
  }
}

__global__ void __launch_bounds__(BATCH_MAX_THREADS) batch_kernel(const __grid_constant__ BatchParams p) {
  BfsCtl *c = p.ctl;
  u64 W = 0, N = 0, edges = 0, push_levels = 0;
  bseed(p, &W, &N);
  if (!bbarrier(c, p.nblocks, p.time_limit_ns)) return;
  u32 level = 0;
  for (;; level++) {
    const u32 cur = level % 3, nxt = (level + 1) % 3, old = (level + 2) % 3;
    const int lp = level & 1;
    u64 n_cur = *(volatile unsigned long long *)&c->n_list[cur];
    if (n_cur > p.list_cap) n_cur = p.list_cap;
    if (n_cur == 0) break;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      c->n_list[old] = 0;
      c->cursor[old] = 0;
      c->spill_count[old] = 0;
      c->spill_cursor[old] = 0;
      if (level < (u32)TRACE_LEVELS) {
        c->trace_t[level] = globaltimer_ns();
        c->trace_n[level] = n_cur;
        c->trace_mode[level] = 1u;
      }
      push_levels++;
    }
    bpush(p, lp, cur, nxt, n_cur, &edges);
    if (!bbarrier(c, p.nblocks, p.time_limit_ns)) return;
    if (*(volatile unsigned long long *)&c->spill_count[cur] != 0) {
      bspill(p, lp, cur, nxt, &edges);
      if (!bbarrier(c, p.nblocks, p.time_limit_ns)) return;
    }
    bcommit(p, lp, nxt, &W, &N);
    if (!bbarrier(c, p.nblocks, p.time_limit_ns)) return;
  }
  W = warp_sum(W);
  N = warp_sum(N);
  edges = warp_sum(edges);
  if (lane_id() == 0) {
    if (W) atomicAdd(&c->stats[ST_W], W);
    if (N) atomicAdd(&c->stats[ST_N], N);
    if (edges) atomicAdd(&c->stats[ST_GROUP_EDGES], edges);
    if (N) atomicAdd(&c->stats[ST_GROUP_VERTICES], N);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c->levels = level;
    c->stats[ST_PUSH_LEVELS] += push_levels;
    c->trace_t[level < (u32)TRACE_LEVELS ? level : TRACE_LEVELS] = globaltimer_ns();
  }
}

// Emission: chunk c (BEMIT_WORDS words = BEMIT_WORDS * 64 vertices) of query
// i's result bitmap (OR of its accepting states' bitmaps).
constexpr int BEMIT_WORDS = 256;

struct BEmitParams {
  const u64 *vis;
  const u64 *vis_off;
  const QueryDesc *qd;
  u64 wps;
  u32 chunks;
  u32 *cnt;
  const u64 *off;
  u32 *rows;  // (query, vertex) pairs
  u64 *digest;
  u32 qbase;  // index of this launch's first query in the caller's arrays
  u64 *qstats;      // optional: per query (rows, digest sum, digest xor) over (source, y)
  const u32 *srcs;  // the launch's sources (for qstats)
  const u32 *evicted;  // optional: queries whose rows are not emitted here
};

template <bool WRITE>
__global__ void __launch_bounds__(BEMIT_WORDS) batch_emit(const BEmitParams p) {
  const u32 c = blockIdx.x, i = blockIdx.y;
  const u64 k = (u64)c * BEMIT_WORDS + threadIdx.x;
  u64 r = 0;
  const u32 fm_all = (p.evicted && p.evicted[i]) ? 0u : p.qd[i].final_mask;
  if (k < p.wps)
    for (u32 fm = fm_all; fm; fm &= fm - 1) r |= __ldcg(p.vis + p.vis_off[i] + (u64)(__ffs(fm) - 1) * p.wps + k);
  const u32 pc = __popcll(r);
  __shared__ u32 warp_tot[BEMIT_WORDS / 32];
  u32 inc = pc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    u32 t = __shfl_up_sync(FULL_MASK, inc, o);
    if (lane_id() >= (u32)o) inc += t;
  }
  if (lane_id() == 31) warp_tot[threadIdx.x >> 5] = inc;
  __syncthreads();
  u32 before = 0, block_tot = 0;
  for (u32 wv = 0; wv < BEMIT_WORDS / 32; wv++) {
    if (wv < (threadIdx.x >> 5)) before += warp_tot[wv];
    block_tot += warp_tot[wv];
  }
  if (!WRITE) {
    u64 hs = 0, hx = 0;
    for (u64 b = r; b; b &= b - 1) {
      u64 h = splitmix64(((u64)(p.qbase + i) << 32) | (k * 64 + __ffsll(b) - 1));
      hs += h;
      hx ^= h;
    }
    hs = warp_sum(hs);
    hx = warp_xor(hx);
    if (lane_id() == 0 && (hs | hx)) {
      atomicAdd(&p.digest[0], hs);
      atomicXor(&p.digest[1], hx);
    }
    if (threadIdx.x == 0) p.cnt[(u64)i * p.chunks + c] = block_tot;
    if (p.qstats) {
      // the same rows as a single-source result: (source, y) pairs
      const u64 s = p.srcs[i];
      u64 qs = 0, qx = 0;
      for (u64 b = r; b; b &= b - 1) {
        u64 h = splitmix64((s << 32) | (k * 64 + __ffsll(b) - 1));
        qs += h;
        qx ^= h;
      }
      qs = warp_sum(qs);
      qx = warp_xor(qx);
      if (lane_id() == 0 && (qs | qx)) {
        atomicAdd(&p.qstats[3 * (u64)i + 1], qs);
        atomicXor(&p.qstats[3 * (u64)i + 2], qx);
      }
      if (threadIdx.x == 0 && block_tot) atomicAdd(&p.qstats[3 * (u64)i], (u64)block_tot);
    }
  } else {
    u64 pos = p.off[(u64)i * p.chunks + c] + before + inc - pc;
    for (u64 b = r; b; b &= b - 1) {
      p.rows[2 * pos] = p.qbase + i;
      p.rows[2 * pos + 1] = (u32)(k * 64 + __ffsll(b) - 1);
      pos++;
    }
  }
}

int berr(rpq_ctx *ctx, cudaError_t e, const char *what) {
  return ctx_error(ctx, RPQ_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <typename T>
struct DBuf {
  rpq_ctx *ctx = nullptr;
  T *p = nullptr;
  uint64_t n = 0;
  int alloc(rpq_ctx *c, uint64_t count) {
    ctx = c;
    n = std::max<uint64_t>(count, 1);
    return ctx_alloc(c, (void **)&p, n * sizeof(T));
  }
  T *release_ownership() {
    T *q = p;
    p = nullptr;
    return q;
  }
  ~DBuf() {
    if (p) ctx_free(ctx, p, n * sizeof(T));
  }
};

}  // namespace

BatchTuning batch_default_tuning() {
  return BatchTuning{BATCH_THREADS, 4096, 1ull << 28, SPILL_CAP, 1ull << 16, false, 4};
}

// One launch over queries [0, nq) of the arrays; appends rows to `out`.
static int batch_launch(rpq_ctx *ctx, const rpq_graph *g, uint32_t qbase, uint32_t nq,
                        const rpq_query *const *queries, const uint32_t *sources, bool materialize,
                        const BatchTuning &tun, BatchOut *out) {
  const DevGraph &dg = graph_dev(g);
  cudaStream_t st = ctx_stream(ctx);
  const u64 wps = ((u64)dg.n + 63) / 64;
  std::vector<QueryDesc> descs(nq);
  std::vector<u64> voff(nq + 1, 0);
  for (uint32_t i = 0; i < nq; i++) {
    descs[i] = query_host(queries[i]).d;
    voff[i + 1] = voff[i] + (u64)descs[i].n_states * wps;
  }
  const u64 vis_words = std::max<u64>(voff[nq], 1);
  DBuf<QueryDesc> d_qd;
  DBuf<u64> d_voff, d_vis, d_l0, d_l1, d_spill, d_small, d_off, d_tmp;
  DBuf<u32> d_src, d_cnt;
  DBuf<BfsCtl> d_ctl;
  int rc;
  if ((rc = d_qd.alloc(ctx, nq)) || (rc = d_voff.alloc(ctx, nq + 1)) || (rc = d_src.alloc(ctx, nq)) ||
      (rc = d_vis.alloc(ctx, vis_words)) || (rc = d_l0.alloc(ctx, tun.list_cap)) ||
      (rc = d_l1.alloc(ctx, tun.list_cap)) || (rc = d_spill.alloc(ctx, SPILL_CAP * 2)) ||
      (rc = d_ctl.alloc(ctx, 1)) || (rc = d_small.alloc(ctx, 4)))
    return rc;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(d_qd.p, descs.data(), nq * sizeof(QueryDesc), cudaMemcpyHostToDevice, st)) ||
      (e = cudaMemcpyAsync(d_voff.p, voff.data(), (nq + 1) * 8, cudaMemcpyHostToDevice, st)) ||
      (e = cudaMemcpyAsync(d_src.p, sources, nq * 4, cudaMemcpyHostToDevice, st)) ||
      (e = cudaMemsetAsync(d_vis.p, 0, vis_words * 8, st)) || (e = cudaMemsetAsync(d_ctl.p, 0, sizeof(BfsCtl), st)) ||
      (e = cudaMemsetAsync(d_small.p, 0, 32, st)))
    return berr(ctx, e, "batch upload");

  const bool evict = out->per_query && !materialize && tun.evict_at > 0;
  DBuf<u64> d_qn, d_qw;
  DBuf<u32> d_ev;
  if (evict) {
    if ((rc = d_qn.alloc(ctx, nq)) || (rc = d_qw.alloc(ctx, nq)) || (rc = d_ev.alloc(ctx, nq))) return rc;
    if ((e = cudaMemsetAsync(d_qn.p, 0, 8ull * nq, st)) || (e = cudaMemsetAsync(d_qw.p, 0, 8ull * nq, st)) ||
        (e = cudaMemsetAsync(d_ev.p, 0, 4ull * nq, st)))
      return berr(ctx, e, "batch counters");
  }
  BatchParams p;
  std::memset(&p, 0, sizeof(p));
  p.qn = evict ? d_qn.p : nullptr;
  p.qw = evict ? d_qw.p : nullptr;
  p.evicted = evict ? d_ev.p : nullptr;
  p.evict_at = evict ? tun.evict_at : 0;
  p.out_off = dg.out_off;
  p.out_col = dg.out_col;
  p.n = dg.n;
  p.L = dg.L;
  p.nq = nq;
  p.qd = d_qd.p;
  p.vis_off = d_voff.p;
  p.srcs = d_src.p;
  p.vis = d_vis.p;
  p.vis_words = vis_words;
  p.m = dg.m;
  p.wps = wps;
  p.list0 = d_l0.p;
  p.list1 = d_l1.p;
  p.list_cap = tun.list_cap;
  p.spill = d_spill.p;
  p.spill_cap = tun.spill_cap;
  p.ctl = d_ctl.p;
  p.time_limit_ns = ctx_time_limit_ns(ctx);
  int bpsm = 0, sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpsm, batch_kernel, tun.threads, 0)) != cudaSuccess)
    return berr(ctx, e, "occupancy");
  const int blocks = std::max(1, std::min(sms, ctx_sm_share(ctx))) * bpsm;
  p.nblocks = (unsigned)blocks;
  // segments only when the unused tails (at most three appending phases per
  // level, one segment per warp each) stay a small part of the list
  const u64 nwarps = (u64)blocks * tun.threads / 32;
  p.append_seg = tun.list_cap >= 16 * 3 * nwarps * APPEND_SEG ? APPEND_SEG : 0;
  void *args[] = {(void *)&p};
  cudaEvent_t ev0, ev1;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  cudaEventRecord(ev0, st);
  e = cudaLaunchCooperativeKernel((void *)batch_kernel, blocks, tun.threads, args, 0, st);
  cudaEventRecord(ev1, st);
  if (e != cudaSuccess) {
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    return berr(ctx, e, "batch_kernel");
  }
  out->stats.launches += 1;
  out->stats.bfs_launches += 1;

  // emission pass 1: counts and digest
  const u32 chunks = (u32)((wps + BEMIT_WORDS - 1) / BEMIT_WORDS);
  const u64 ncnt = (u64)nq * chunks;
  if ((rc = d_cnt.alloc(ctx, ncnt)) || (rc = d_off.alloc(ctx, ncnt)) || (rc = d_tmp.alloc(ctx, scan_tmp_words(ncnt))))
    return rc;
  BEmitParams ep;
  ep.vis = d_vis.p;
  ep.vis_off = d_voff.p;
  ep.qd = d_qd.p;
  ep.wps = wps;
  ep.chunks = chunks;
  ep.cnt = d_cnt.p;
  ep.off = d_off.p;
  ep.rows = nullptr;
  ep.digest = d_small.p;
  ep.qbase = qbase;
  ep.srcs = d_src.p;
  ep.qstats = nullptr;
  ep.evicted = evict ? d_ev.p : nullptr;
  DBuf<u64> d_qstats;
  if (out->per_query) {
    if ((rc = d_qstats.alloc(ctx, 3ull * nq))) return rc;
    if ((e = cudaMemsetAsync(d_qstats.p, 0, 24ull * nq, st)) != cudaSuccess) return berr(ctx, e, "memset");
    ep.qstats = d_qstats.p;
  }
  dim3 grid(chunks, nq);
  batch_emit<false><<<grid, BEMIT_WORDS, 0, st>>>(ep);
  if ((e = cudaGetLastError()) != cudaSuccess) return berr(ctx, e, "batch_emit");
  if ((e = exclusive_scan_u32_to_u64(d_cnt.p, d_off.p, ncnt, d_small.p + 2, d_tmp.p, st)) != cudaSuccess)
    return berr(ctx, e, "scan");
  out->stats.launches += 2;
  BfsCtl hctl;
  u64 hsmall[3];
  if ((e = cudaMemcpyAsync(&hctl, d_ctl.p, sizeof(BfsCtl), cudaMemcpyDeviceToHost, st)) ||
      (e = cudaMemcpyAsync(hsmall, d_small.p, 24, cudaMemcpyDeviceToHost, st)) || (e = cudaStreamSynchronize(st))) {
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    return berr(ctx, e, "batch readback");
  }
  float ms = 0;
  cudaEventElapsedTime(&ms, ev0, ev1);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  if (hctl.err == ERR_LIST_FULL) return RPQ_BATCH_SPLIT;
  std::vector<u64> hqn, hqw;
  std::vector<u32> hev;
  if (out->per_query && hctl.err == 0) {
    std::vector<u64> qs(3ull * nq);
    if ((e = cudaMemcpy(qs.data(), d_qstats.p, 24ull * nq, cudaMemcpyDeviceToHost)) != cudaSuccess)
      return berr(ctx, e, "qstats");
    out->qstats.insert(out->qstats.end(), qs.begin(), qs.end());
    if (evict) {
      hqn.resize(nq);
      hqw.resize(nq);
      hev.resize(nq);
      if ((e = cudaMemcpy(hqn.data(), d_qn.p, 8ull * nq, cudaMemcpyDeviceToHost)) ||
          (e = cudaMemcpy(hqw.data(), d_qw.p, 8ull * nq, cudaMemcpyDeviceToHost)) ||
          (e = cudaMemcpy(hev.data(), d_ev.p, 4ull * nq, cudaMemcpyDeviceToHost)))
        return berr(ctx, e, "batch counters");
    }
  }
  if (hctl.err >= ERR_BOUNDS)
    return ctx_error(ctx, RPQ_ERR_CUDA, "batch traversal index check " + std::to_string(hctl.err - ERR_BOUNDS) +
                                            " failed (a device index out of its array; access skipped)");
  if (hctl.err) return ctx_error(ctx, RPQ_ERR_TIMEOUT, "batch traversal grid barrier wait ran out of time");
  if (ctx_trace(ctx)) {
    const uint32_t nl = (uint32_t)std::min<u64>(hctl.levels, TRACE_LEVELS);
    std::fprintf(stderr, "[rpq trace] batch nq=%u threads=%d blocks=%d levels=%llu W=%llu N=%llu %.3f ms\n", nq,
                 tun.threads, blocks, (unsigned long long)hctl.levels, (unsigned long long)hctl.stats[ST_W],
                 (unsigned long long)hctl.stats[ST_N], ms);
    for (uint32_t l = 0; l < nl; l++)
      std::fprintf(stderr, "[rpq trace]   level %3u n=%10llu %9.3f ms\n", l, (unsigned long long)hctl.trace_n[l],
                   (hctl.trace_t[l + 1] - hctl.trace_t[l]) * 1e-6);
  }
  out->stats.bfs_ms += ms;
  if (evict) {
    // exact work of the queries that stayed; evicted ones are counted by their
    // multi-source evaluation
    for (uint32_t i = 0; i < nq; i++) {
      if (hev[i]) {
        out->evicted_idx.push_back(qbase + i);
        continue;
      }
      out->stats.product_edges += hqw[i];
      out->stats.product_vertices += hqn[i];
    }
  } else {
    out->stats.product_edges += hctl.stats[ST_W];
    out->stats.product_vertices += hctl.stats[ST_N];
  }
  out->stats.levels += hctl.levels;
  out->stats.push_levels += hctl.stats[ST_PUSH_LEVELS];
  out->stats.group_edges += hctl.stats[ST_GROUP_EDGES];
  out->stats.group_vertices += hctl.stats[ST_GROUP_VERTICES];
  out->stats.lane_groups += 1;
  const u64 total = hsmall[2];
  out->count += total;
  out->dsum += hsmall[0];
  out->dxor ^= hsmall[1];
  if (materialize && total) {
    u32 *rows = nullptr;
    if ((rc = ctx_alloc(ctx, (void **)&rows, total * 8))) return rc;
    ep.rows = rows;
    batch_emit<true><<<grid, BEMIT_WORDS, 0, st>>>(ep);
    if ((e = cudaGetLastError()) != cudaSuccess) {
      ctx_free(ctx, rows, total * 8);
      return berr(ctx, e, "batch_emit");
    }
    out->stats.launches += 1;
    out->chunks.push_back({rows, total});
  }
  return RPQ_OK;
}

int batch_run(rpq_ctx *ctx, const rpq_graph *g, uint32_t nq, const rpq_query *const *queries,
              const uint32_t *sources, bool materialize, const BatchTuning &tun, BatchOut *out) {
  for (uint32_t b0 = 0; b0 < nq;) {
    uint32_t k = std::min<uint32_t>(tun.queries_per_launch, nq - b0);
    for (;;) {
      int rc = batch_launch(ctx, g, b0, k, queries + b0, sources + b0, materialize, tun, out);
      if (rc == RPQ_OK) break;
      if (rc != RPQ_BATCH_SPLIT) return rc;
      if (k == 1) return ctx_error(ctx, RPQ_ERR_OUT_OF_BUDGET, "one query's frontier exceeds the list capacity");
      k = (k + 1) / 2;  // frontier list too small for this many queries at once: halve
    }
    b0 += k;
  }
  if (!out->per_query) return RPQ_OK;
  // Queries that left the batch, grouped by automaton, are evaluated by the
  // direction-optimizing multi-source engine with every lane's own row count
  // and digest (work items below).
  std::map<std::string, std::vector<uint32_t>> groups;
  for (uint32_t i : out->evicted_idx) {
    const QueryDesc &d = query_host(queries[i]).d;
    groups[std::string(reinterpret_cast<const char *>(&d), sizeof(d))].push_back(i);
  }
  // Work items, run side by side on helper contexts (own streams, a share of
  // the SMs each), one host thread per helper taking items in turn:
  //   * an automaton with more than 64 evicted queries: one bit-sliced launch
  //     over its start vertices (256 lanes per word);
  //   * smaller ones: units of one automaton and at most 64 start vertices,
  //     16 units per multi-automaton launch (each unit a lane group running
  //     its own automaton).
  // One lane per query, in source order (a repeated start vertex gets a lane
  // of its own, so the work counter stays the sum over queries).
  struct Item {
    std::vector<uint32_t> single;               // query indices, one automaton
    std::vector<std::vector<uint32_t>> units;   // query indices per unit
  };
  std::vector<Item> todo;
  Item pending;
  for (auto &kv : groups) {
    std::vector<uint32_t> members = kv.second;
    std::sort(members.begin(), members.end(),
              [&](uint32_t a, uint32_t b) { return sources[a] < sources[b] || (sources[a] == sources[b] && a < b); });
    if (members.size() > 64 || !tun.multi) {
      Item it;
      it.single = members;
      todo.push_back(std::move(it));
      continue;
    }
    pending.units.push_back(members);
    if (pending.units.size() == 16) {
      todo.push_back(std::move(pending));
      pending = Item();
    }
  }
  if (!pending.units.empty()) todo.push_back(std::move(pending));
  const int k = (int)std::min<size_t>(std::max(1u, std::min(tun.streams, MAX_REGROUP_STREAMS)), todo.size());
  std::vector<rpq_ctx *> helpers;
  int rc = k > 1 ? ctx_helpers(ctx, k, &helpers) : RPQ_OK;
  if (rc) return rc;
  if (k <= 1) helpers.assign(1, ctx);
  std::atomic<size_t> next{0};
  std::vector<int> rcs(helpers.size(), RPQ_OK);
  std::vector<rpq_stats> hst(helpers.size());
  std::vector<uint64_t> launches(helpers.size(), 0);
  auto assign = [&](const std::vector<uint32_t> &tasks, const std::vector<uint64_t> &ls, size_t at) {
    for (size_t j = 0; j < tasks.size(); j++)
      for (int c = 0; c < 3; c++) out->qstats[3ull * tasks[j] + c] = ls[3 * (at + j) + c];
  };
  auto run_single = [&](size_t h, const std::vector<uint32_t> &tasks) {
    std::vector<uint32_t> srcs;
    for (uint32_t i : tasks) srcs.push_back(sources[i]);
    std::vector<uint64_t> ls;
    int r = rpq_lane_stats_for_sources(helpers[h], g, queries[tasks[0]], srcs, &ls, &hst[h]);
    if (r == RPQ_OK) {
      assign(tasks, ls, 0);
      launches[h]++;
    }
    return r;
  };
  auto work = [&](size_t h) {
    std::memset(&hst[h], 0, sizeof(rpq_stats));
    cudaSetDevice(ctx_device(ctx));
    for (size_t t; (t = next.fetch_add(1)) < todo.size();) {
      const Item &it = todo[t];
      int r = RPQ_OK;
      if (!it.single.empty()) {
        r = run_single(h, it.single);
      } else {
        std::vector<MultiUnit> units(it.units.size());
        for (size_t u = 0; u < it.units.size(); u++) {
          units[u].q = queries[it.units[u][0]];
          for (uint32_t i : it.units[u]) units[u].srcs.push_back(sources[i]);
        }
        std::vector<uint64_t> ls;
        r = rpq_lane_stats_multi(helpers[h], g, units, &ls, &hst[h]);
        if (r == RPQ_OK) {
          size_t at = 0;
          for (const auto &tasks : it.units) {
            assign(tasks, ls, at);
            at += tasks.size();
          }
          launches[h]++;
        } else if (r == RPQ_ERR_TOO_COMPLEX) {
          // the union of these automata does not fit a descriptor: one launch each
          r = RPQ_OK;
          for (size_t u = 0; u < it.units.size() && r == RPQ_OK; u++) r = run_single(h, it.units[u]);
        }
      }
      if (r) {
        rcs[h] = r;
        next = todo.size();
        return;
      }
    }
  };
  std::vector<std::thread> threads;
  for (size_t h = 1; h < helpers.size(); h++) threads.emplace_back(work, h);
  work(0);
  for (auto &t : threads) t.join();
  for (size_t h = 0; h < helpers.size(); h++) {
    if (rcs[h]) return ctx_error(ctx, rcs[h], "multi-source evaluation of evicted queries failed");
    rpq_stats &a = out->stats, &b = hst[h];
    a.product_edges += b.product_edges;
    a.product_vertices += b.product_vertices;
    a.levels += b.levels;
    a.push_levels += b.push_levels;
    a.pull_levels += b.pull_levels;
    a.bfs_ms += b.bfs_ms;
    a.emit_ms += b.emit_ms;
    a.bfs_launches += b.bfs_launches;
    a.launches += b.launches;
    a.alg_bytes += b.alg_bytes;
    a.group_product_edges += b.group_product_edges;
    a.group_label_rows += b.group_label_rows;
    out->regroup_launches += launches[h];
  }
  out->evicted += out->evicted_idx.size();
  out->stats.evicted += out->evicted_idx.size();
  // with per-query summaries the totals are theirs: rows and digests of the
  // (source, y) rows every query would report alone
  out->count = out->dsum = out->dxor = 0;
  for (size_t i = 0; 3 * i + 2 < out->qstats.size(); i++) {
    out->count += out->qstats[3 * i];
    out->dsum += out->qstats[3 * i + 1];
    out->dxor ^= out->qstats[3 * i + 2];
  }
  return RPQ_OK;
}

}  // namespace rpq
