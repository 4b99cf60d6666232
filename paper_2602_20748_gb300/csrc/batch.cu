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
  // Visited representation.  hash_bits == 0: dense bitmaps (vis, vis_off).
  // Otherwise query i owns an open-addressing table of 2^hash_bits slots at
  // vis + (i << hash_bits), keys (state << 32 | vertex) + 1 (0 = free), and a
  // result table of the same size at rtab + (i << hash_bits), keys vertex + 1;
  // a row found the first time is counted and digested at once into
  // qstats[3 i ..] (rows, digest sum, digest xor of (source, y)).  A query
  // whose table has no free slot within HASH_PROBES of a key's home leaves
  // the batch (evicted).
  u32 hash_bits;
  u64 *rtab;
  unsigned long long *qstats;
  // serving: per query (slot), the last level whose list holds entries of it
  // (the commit stamps it); nullptr in batches
  u32 *active;
};

constexpr u32 HASH_PROBES = 32;

__device__ __forceinline__ u32 hslot(u64 key, u32 bits) {
  return (u32)((key * 0x9E3779B97F4A7C15ull) >> (64 - bits));
}

// Inserts key into the table of 2^bits slots at tab: 1 = inserted by this
// thread, 0 = already there, -1 = no free slot near its home.
__device__ __forceinline__ int hinsert(u64 *tab, u32 bits, u64 key) {
  const u32 mask = (1u << bits) - 1u;
  u32 h = hslot(key, bits);
  for (u32 probe = 0; probe < HASH_PROBES; probe++, h = (h + 1) & mask) {
    const u64 cur = __ldcg(tab + h);
    if (cur == key) return 0;
    if (cur == 0) {
      const u64 old = atomicCAS((unsigned long long *)(tab + h), 0ull, (unsigned long long)key);
      if (old == 0) return 1;
      if (old == key) return 0;
    }
  }
  return -1;
}

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
  if (p.hash_bits) {
    if (bad(p, q2 >= p.qd[i].n_states, 3)) return false;
    const int r = hinsert(p.vis + ((u64)i << p.hash_bits), p.hash_bits, (((u64)q2 << 32) | w) + 1);
    if (r < 0) p.evicted[i] = 1u;  // table full: the query leaves the batch
    if (r <= 0) return false;
    if ((p.qd[i].final_mask >> q2) & 1u) {
      // a row (source, w) the first time: count and digest it now
      const int rr = hinsert(p.rtab + ((u64)i << p.hash_bits), p.hash_bits, (u64)w + 1);
      if (rr < 0) p.evicted[i] = 1u;
      if (rr > 0) {
        const u64 h = splitmix64(((u64)p.srcs[i] << 32) | w);
        atomicAdd(&p.qstats[3 * (u64)i], 1ull);
        atomicAdd(&p.qstats[3 * (u64)i + 1], h);
        atomicXor(&p.qstats[3 * (u64)i + 2], h);
      }
    }
    return true;
  }
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

__device__ void bcommit(const BatchParams &p, int lp, u32 nxt, u64 *W, u64 *N, u32 stamp = 0) {
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
      if (ok && p.active) p.active[i] = stamp;
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

// ---------------------------------------------------------------------------
// Persistent serving launch: the batched engine over slots instead of a fixed
// query list.  A slot is a query in flight (descriptor, source, hash tables,
// counters); requests are admitted into free slots at every level boundary.
// ---------------------------------------------------------------------------
struct ServeState {              // device memory, kept across launches
  unsigned int free_top;         // free slot ids are free_stack[0 .. free_top)
  unsigned int busy;             // slots in service
  unsigned int admit_k;          // requests the next admission phase takes
  unsigned int exit;             // 1: the launch ends at the top of the next level
  unsigned long long head;       // requests taken from the ring
  unsigned long long done_count; // replies written to the ring
  unsigned long long admitted;   // requests admitted over all launches
};

struct ServeParams {
  BatchParams b;                 // slots as queries (b.nq slots, hash mode)
  ServeShared *sh;               // mapped host memory
  const ServeReq *reqs;          // mapped request ring
  ServeDone *dones;              // mapped reply ring
  u32 ring;                      // entries per ring (a power of two)
  u32 admit_max;                 // requests admitted per level at most
  u32 *slot_src;                 // = b.srcs, writable
  QueryDesc *slot_qd;            // = b.qd, writable
  u32 *free_stack;
  u32 *busy;                     // per slot: 1 while in service
  unsigned long long *tickets;   // per slot
  ServeState *st;
};

// Block 0, thread 0, between phases: publish the replies written so far and
// decide what the next admission phase takes, or that the launch ends.
__device__ void serve_decide(const ServeParams &sp) {
  ServeState *st = sp.st;
  __threadfence_system();
  sp.sh->done_tail = st->done_count;
  const u64 tail = sp.sh->req_tail, dh = sp.sh->done_head;
  const u64 pending = tail - st->head;
  // every admitted request gets one reply: keep room for the replies of all
  // slots in service plus the new ones
  const u64 unread = st->done_count - dh;
  const u64 room = (u64)sp.ring > unread + st->busy ? (u64)sp.ring - unread - st->busy : 0;
  u64 k = min(min(pending, (u64)st->free_top), min(room, (u64)sp.admit_max));
  if (sp.sh->stop) k = 0;
  st->admit_k = (unsigned)k;
  st->exit = (st->busy == 0 && k == 0) ? 1u : 0u;
}

// Admission: warp w takes request head + w into slot free_stack[top - 1 - w],
// copies its descriptor, resets the slot's counters and seeds (source, start
// state) into the current list.
__device__ void serve_admit(const ServeParams &sp, u32 level, u32 cur, int lp, u64 *W, u64 *N) {
  const BatchParams &p = sp.b;
  const ServeState *st = sp.st;
  const u32 k = *(volatile const unsigned *)&st->admit_k;
  const u64 head = *(volatile const unsigned long long *)&st->head;
  const u32 top = *(volatile const unsigned *)&st->free_top;
  const u32 lane = lane_id();
  const u64 warp = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
  u64 *list = lp ? p.list1 : p.list0;
  BAppender app;
  // warp-uniform loop: every lane of a warp takes the same requests
  for (u64 w = warp; w < k; w += nwarps) {
    const ServeReq *rq = sp.reqs + ((head + w) & (u64)(sp.ring - 1));
    const u32 slot = sp.free_stack[top - 1 - (u32)w];
    bool take = false;
    u32 src = 0;
    if (!bad(p, slot >= p.nq, 20)) {
      const unsigned *from = reinterpret_cast<const unsigned *>(&rq->qd);
      unsigned *to = reinterpret_cast<unsigned *>(sp.slot_qd + slot);
      for (u32 j = lane; j < sizeof(QueryDesc) / 4; j += 32) to[j] = *(volatile const unsigned *)(from + j);
      src = *(volatile const unsigned *)&rq->source;
      if (lane == 0) {
        sp.slot_src[slot] = src;
        sp.tickets[slot] = *(volatile const unsigned long long *)&rq->ticket;
        p.qn[slot] = 0;
        p.qw[slot] = 0;
        p.evicted[slot] = 0;
        p.qstats[3 * (u64)slot] = 0;
        p.qstats[3 * (u64)slot + 1] = 0;
        p.qstats[3 * (u64)slot + 2] = 0;
        p.active[slot] = level;
        sp.busy[slot] = 1;
      }
      __syncwarp();
      if (lane == 0 && src < p.n && sp.slot_qd[slot].n_states > 0) {
        take = bvisit(p, slot, 0, src);
        if (take) {
          const u32 d = bdegsum(p, sp.slot_qd[slot], 0, src);
          p.qn[slot] = 1;
          p.qw[slot] = d;
          *W += d;
          *N += 1;
        }
      }
    }
    bappend(p, app, take, bentry(slot, 0, src), &p.ctl->n_list[cur], list);
  }
  bappend_close(p, app, list);
}

// Retirement: a warp per busy slot whose frontier ran empty (no entry of it
// in the next list) writes its reply, clears its hash tables and frees the
// slot.  An evicted query stops expanding, so its slot is retired (with the
// evicted mark) one level later, once no list holds entries of it any more:
// a slot reused sooner would inherit them.
__device__ void serve_retire(const ServeParams &sp, u32 level) {
  const BatchParams &p = sp.b;
  ServeState *st = sp.st;
  const u32 lane = lane_id();
  const u64 warp = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
  const u64 tsize = 1ull << p.hash_bits;
  for (u64 s0 = warp; s0 < p.nq; s0 += nwarps) {
    const u32 s = (u32)s0;
    bool fin = false;
    if (lane == 0) fin = __ldcg(sp.busy + s) && __ldcg(p.active + s) <= level;
    fin = __shfl_sync(FULL_MASK, fin, 0);
    if (!fin) continue;
    if (lane == 0) {
      const u64 idx = atomicAdd(&st->done_count, 1ull);
      ServeDone *d = sp.dones + (idx & (u64)(sp.ring - 1));
      d->ticket = sp.tickets[s];
      d->count = __ldcg(p.qstats + 3 * (u64)s);
      d->dsum = __ldcg(p.qstats + 3 * (u64)s + 1);
      d->dxor = __ldcg(p.qstats + 3 * (u64)s + 2);
      d->product_vertices = __ldcg(p.qn + s);
      d->product_edges = __ldcg(p.qw + s);
      d->evicted = __ldcg(p.evicted + s) ? 1u : 0u;
      __threadfence_system();
    }
    // the slot's visited and result tables back to empty
    ulonglong2 *vt = reinterpret_cast<ulonglong2 *>(p.vis + s0 * tsize);
    ulonglong2 *rt = reinterpret_cast<ulonglong2 *>(p.rtab + s0 * tsize);
    for (u64 j = lane; j < tsize / 2; j += 32) {
      vt[j] = make_ulonglong2(0, 0);
      rt[j] = make_ulonglong2(0, 0);
    }
    __syncwarp();
    if (lane == 0) {
      sp.busy[s] = 0;
      sp.free_stack[atomicAdd(&st->free_top, 1u)] = s;
      atomicSub(&st->busy, 1u);
    }
  }
}

__global__ void __launch_bounds__(BATCH_MAX_THREADS) serve_kernel(const __grid_constant__ ServeParams sp) {
  const BatchParams &p = sp.b;
  BfsCtl *c = p.ctl;
  ServeState *st = sp.st;
  u64 W = 0, N = 0, edges = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) serve_decide(sp);
  if (!bbarrier(c, p.nblocks, p.time_limit_ns)) return;
  u32 level = 0;
  for (;; level++) {
    const u32 cur = level % 3, nxt = (level + 1) % 3, old = (level + 2) % 3;
    const int lp = level & 1;
    if (*(volatile unsigned *)&st->exit) break;
    serve_admit(sp, level, cur, lp, &W, &N);
    if (!bbarrier(c, p.nblocks, p.time_limit_ns)) return;
    u64 n_cur = *(volatile unsigned long long *)&c->n_list[cur];
    if (n_cur > p.list_cap) n_cur = p.list_cap;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      // the admitted requests left the ring and the free stack
      const u32 k = st->admit_k;
      st->free_top -= k;
      st->busy += k;
      st->head += k;
      st->admitted += k;
      sp.sh->req_head = st->head;
      c->n_list[old] = 0;
      c->cursor[old] = 0;
      c->spill_count[old] = 0;
      c->spill_cursor[old] = 0;
      if (level < (u32)TRACE_LEVELS) {
        c->trace_t[level] = globaltimer_ns();
        c->trace_n[level] = n_cur;
        c->trace_mode[level] = 1u;
      }
    }
    if (n_cur > 0) {
      bpush(p, lp, cur, nxt, n_cur, &edges);
      if (!bbarrier(c, p.nblocks, p.time_limit_ns)) return;
      if (*(volatile unsigned long long *)&c->spill_count[cur] != 0) {
        bspill(p, lp, cur, nxt, &edges);
        if (!bbarrier(c, p.nblocks, p.time_limit_ns)) return;
      }
      bcommit(p, lp, nxt, &W, &N, level + 1);
      if (!bbarrier(c, p.nblocks, p.time_limit_ns)) return;
    }
    serve_retire(sp, level);
    if (!bbarrier(c, p.nblocks, p.time_limit_ns)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) serve_decide(sp);
    if (!bbarrier(c, p.nblocks, p.time_limit_ns)) return;
  }
  W = warp_sum(W);
  N = warp_sum(N);
  edges = warp_sum(edges);
  if (lane_id() == 0) {
    if (W) atomicAdd(&c->stats[ST_W], W);
    if (N) atomicAdd(&c->stats[ST_N], N);
    if (edges) atomicAdd(&c->stats[ST_GROUP_EDGES], edges);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) c->levels = level;
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
  return BatchTuning{BATCH_THREADS, 4096, 1ull << 28, SPILL_CAP, 1ull << 16, false, 4, 4096, false, false};
}

// One launch over queries [0, nq) of the arrays; appends rows to `out`.
static int batch_launch(rpq_ctx *ctx, const rpq_graph *g, uint32_t qbase, uint32_t nq,
                        const rpq_query *const *queries, const uint32_t *sources, bool materialize,
                        const BatchTuning &tun, BatchOut *out) {
  const DevGraph &dg = graph_dev(g);
  cudaStream_t st = ctx_stream(ctx);
  const u64 wps = ((u64)dg.n + 63) / 64;
  // hash tables only for per-query summaries (their rows are counted as they
  // are found), sized for twice the eviction threshold
  const bool use_hash = tun.hash && out->per_query && !materialize;
  uint32_t hbits = 0;
  if (use_hash) {
    const u64 cap = std::max<u64>(64, 2 * (tun.evict_at ? tun.evict_at : 4096));
    while ((1ull << hbits) < cap) hbits++;
  }
  std::vector<QueryDesc> descs(nq);
  std::vector<u64> voff(nq + 1, 0);
  for (uint32_t i = 0; i < nq; i++) {
    descs[i] = query_host(queries[i]).d;
    voff[i + 1] = voff[i] + (use_hash ? (1ull << hbits) : (u64)descs[i].n_states * wps);
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

  const bool evict = out->per_query && !materialize && (tun.evict_at > 0 || use_hash);
  DBuf<u64> d_qn, d_qw, d_rtab, d_hq;
  DBuf<u32> d_ev;
  if (use_hash) {
    if ((rc = d_rtab.alloc(ctx, vis_words)) || (rc = d_hq.alloc(ctx, 3ull * nq))) return rc;
    if ((e = cudaMemsetAsync(d_rtab.p, 0, vis_words * 8, st)) || (e = cudaMemsetAsync(d_hq.p, 0, 24ull * nq, st)))
      return berr(ctx, e, "hash tables");
  }
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
  p.evict_at = evict ? (tun.evict_at ? tun.evict_at : (1ull << hbits) / 2) : 0;
  p.hash_bits = hbits;
  p.rtab = use_hash ? d_rtab.p : nullptr;
  p.qstats = use_hash ? d_hq.p : nullptr;
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

  // emission pass 1: counts and digest (hash mode: rows were counted as they
  // were found, nothing to scan)
  const u32 chunks = use_hash ? 1u : (u32)((wps + BEMIT_WORDS - 1) / BEMIT_WORDS);
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
  if (out->per_query && !use_hash) {
    if ((rc = d_qstats.alloc(ctx, 3ull * nq))) return rc;
    if ((e = cudaMemsetAsync(d_qstats.p, 0, 24ull * nq, st)) != cudaSuccess) return berr(ctx, e, "memset");
    ep.qstats = d_qstats.p;
  }
  dim3 grid(chunks, nq);
  if (!use_hash) {
    batch_emit<false><<<grid, BEMIT_WORDS, 0, st>>>(ep);
    if ((e = cudaGetLastError()) != cudaSuccess) return berr(ctx, e, "batch_emit");
    if ((e = exclusive_scan_u32_to_u64(d_cnt.p, d_off.p, ncnt, d_small.p + 2, d_tmp.p, st)) != cudaSuccess)
      return berr(ctx, e, "scan");
    out->stats.launches += 2;
  }
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
    if ((e = cudaMemcpy(qs.data(), use_hash ? d_hq.p : d_qstats.p, 24ull * nq, cudaMemcpyDeviceToHost)) !=
        cudaSuccess)
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

// ---------------------------------------------------------------------------
// Serving engine (host side)
// ---------------------------------------------------------------------------
constexpr uint32_t SERVE_RING = 8192;       // entries per ring
constexpr uint32_t SERVE_ADMIT_MAX = 2048;  // requests admitted per level at most
constexpr int SERVE_THREADS = 256;

struct ServeEngine {
  rpq_ctx *ctx = nullptr;
  const rpq_graph *g = nullptr;
  uint32_t slots = 0, hbits = 0;
  uint64_t evict_at = 0, list_cap = 0;
  DBuf<QueryDesc> slot_qd;
  DBuf<u32> slot_src, busy, free_stack, evicted, active;
  DBuf<u64> qn, qw, qstats, tickets, vis, rtab, list0, list1, spill;
  DBuf<BfsCtl> ctl;
  DBuf<ServeState> st;
  ServeShared *sh = nullptr;  // mapped host memory (host view)
  ServeReq *reqs = nullptr;
  ServeDone *dones = nullptr;
  void *sh_d = nullptr, *reqs_d = nullptr, *dones_d = nullptr;  // device views
  cudaEvent_t done_ev = nullptr;
  bool running = false;
  int blocks = 0;
  uint64_t launches = 0;
  ServeParams params;                  // fixed for the engine's lifetime
  cudaGraphExec_t graph = nullptr;     // the captured relaunch sequence (nullptr: launched directly)
};

uint64_t serve_engine_bytes(uint32_t slots, uint32_t hash_bits) {
  const uint64_t per_slot = sizeof(QueryDesc) + 4 * 5 + 8 * 6;
  const uint64_t tables = 2ull * ((uint64_t)slots << hash_bits) * 8;
  const uint64_t lists = 2ull * (((uint64_t)slots << hash_bits) + (1ull << 22)) * 8;
  return (uint64_t)slots * per_slot + tables + lists + SPILL_CAP * 16 + sizeof(BfsCtl) + sizeof(ServeState);
}

static int serve_reset_state(ServeEngine *e) {
  cudaStream_t st = ctx_stream(e->ctx);
  std::vector<u32> fs(e->slots);
  for (uint32_t i = 0; i < e->slots; i++) fs[i] = e->slots - 1 - i;
  ServeState h{};
  h.free_top = e->slots;
  h.head = e->sh->req_head;
  h.done_count = e->sh->done_tail;
  const uint64_t tw = (uint64_t)e->slots << e->hbits;
  cudaError_t err;
  if ((err = cudaMemsetAsync(e->vis.p, 0, tw * 8, st)) || (err = cudaMemsetAsync(e->rtab.p, 0, tw * 8, st)) ||
      (err = cudaMemsetAsync(e->busy.p, 0, 4ull * e->slots, st)) ||
      (err = cudaMemsetAsync(e->list0.p, 0, 8, st)) ||
      (err = cudaMemcpyAsync(e->free_stack.p, fs.data(), 4ull * e->slots, cudaMemcpyHostToDevice, st)) ||
      (err = cudaMemcpyAsync(e->st.p, &h, sizeof(h), cudaMemcpyHostToDevice, st)) || (err = cudaStreamSynchronize(st)))
    return berr(e->ctx, err, "serving state reset");
  return RPQ_OK;
}

// The serving launch's parameters: the engine's buffers, fixed for its life.
static void serve_params(ServeEngine *e) {
  ServeParams &sp = e->params;
  std::memset(&sp, 0, sizeof(sp));
  const DevGraph &dg = graph_dev(e->g);
  BatchParams &p = sp.b;
  p.out_off = dg.out_off;
  p.out_col = dg.out_col;
  p.n = dg.n;
  p.L = dg.L;
  p.nq = e->slots;
  p.qd = e->slot_qd.p;
  p.vis_off = nullptr;
  p.srcs = e->slot_src.p;
  p.vis = e->vis.p;
  p.vis_words = (uint64_t)e->slots << e->hbits;
  p.m = dg.m;
  p.wps = 0;
  p.list0 = e->list0.p;
  p.list1 = e->list1.p;
  p.list_cap = e->list_cap;
  p.spill = e->spill.p;
  p.spill_cap = SPILL_CAP;
  p.ctl = e->ctl.p;
  p.nblocks = (unsigned)e->blocks;
  p.time_limit_ns = ctx_time_limit_ns(e->ctx);
  p.qn = e->qn.p;
  p.qw = e->qw.p;
  p.evicted = e->evicted.p;
  p.evict_at = e->evict_at;
  p.append_seg = APPEND_SEG;
  p.hash_bits = e->hbits;
  p.rtab = e->rtab.p;
  p.qstats = e->qstats.p;
  p.active = e->active.p;
  sp.sh = static_cast<ServeShared *>(e->sh_d);
  sp.reqs = static_cast<const ServeReq *>(e->reqs_d);
  sp.dones = static_cast<ServeDone *>(e->dones_d);
  sp.ring = SERVE_RING;
  sp.admit_max = SERVE_ADMIT_MAX;
  sp.slot_src = e->slot_src.p;
  sp.slot_qd = e->slot_qd.p;
  sp.free_stack = e->free_stack.p;
  sp.busy = e->busy.p;
  sp.tickets = e->tickets.p;
  sp.st = e->st.p;
}

// One relaunch: the control block cleared, then the persistent kernel.
static cudaError_t serve_issue(ServeEngine *e, cudaStream_t st) {
  void *args[] = {(void *)&e->params};
  cudaError_t err = cudaMemsetAsync(e->ctl.p, 0, sizeof(BfsCtl), st);
  if (err == cudaSuccess)
    err = cudaLaunchCooperativeKernel((void *)serve_kernel, e->blocks, SERVE_THREADS, args, 0, st);
  return err;
}

// Captures the relaunch sequence in a CUDA graph (instantiated once, launched
// on every relaunch).  If the runtime refuses the capture the engine keeps
// launching directly.
static void serve_capture(ServeEngine *e) {
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  cudaGraph_t graph = nullptr;
  cudaError_t err = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (err == cudaSuccess) {
    const cudaError_t issued = serve_issue(e, cs);
    err = cudaStreamEndCapture(cs, &graph);
    if (issued != cudaSuccess) err = issued;
  }
  if (err == cudaSuccess && graph) err = cudaGraphInstantiate(&e->graph, graph, 0);
  if (err != cudaSuccess) {
    e->graph = nullptr;
    cudaGetLastError();
  }
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
}

int serve_engine_create(rpq_ctx *ctx, const rpq_graph *g, uint32_t slots, uint32_t hash_bits, uint64_t evict_at,
                        ServeEngine **out) {
  *out = nullptr;
  if (slots == 0 || hash_bits < 6 || hash_bits > 24) return ctx_error(ctx, RPQ_ERR_INVALID_ARG, "bad serving sizes");
  auto *e = new ServeEngine;
  e->ctx = ctx;
  e->g = g;
  e->slots = slots;
  e->hbits = hash_bits;
  e->evict_at = std::max<uint64_t>(1, std::min<uint64_t>(evict_at, (1ull << hash_bits) / 2));
  int bpsm = 0, sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpsm, serve_kernel, SERVE_THREADS, 0);
  if (err != cudaSuccess || bpsm <= 0) {
    delete e;
    return ctx_error(ctx, RPQ_ERR_CUDA, "serving kernel occupancy");
  }
  e->blocks = std::max(1, std::min(sms, ctx_sm_share(ctx))) * bpsm;
  const uint64_t nwarps = (uint64_t)e->blocks * SERVE_THREADS / 32;
  // every entry is a first visit of its slot's table, so a list never holds
  // more than slots x table size entries, plus the unused tails of reserved
  // segments (three appending phases per level)
  e->list_cap = ((uint64_t)slots << hash_bits) + 3 * nwarps * APPEND_SEG;
  const uint64_t tw = (uint64_t)slots << hash_bits;
  int rc;
  if ((rc = e->slot_qd.alloc(ctx, slots)) || (rc = e->slot_src.alloc(ctx, slots)) || (rc = e->busy.alloc(ctx, slots)) ||
      (rc = e->free_stack.alloc(ctx, slots)) || (rc = e->evicted.alloc(ctx, slots)) ||
      (rc = e->active.alloc(ctx, slots)) || (rc = e->qn.alloc(ctx, slots)) || (rc = e->qw.alloc(ctx, slots)) ||
      (rc = e->qstats.alloc(ctx, 3ull * slots)) || (rc = e->tickets.alloc(ctx, slots)) ||
      (rc = e->vis.alloc(ctx, tw)) || (rc = e->rtab.alloc(ctx, tw)) || (rc = e->list0.alloc(ctx, e->list_cap)) ||
      (rc = e->list1.alloc(ctx, e->list_cap)) || (rc = e->spill.alloc(ctx, SPILL_CAP * 2)) ||
      (rc = e->ctl.alloc(ctx, 1)) || (rc = e->st.alloc(ctx, 1))) {
    delete e;
    return rc;
  }
  void *h = nullptr;
  const size_t bytes = sizeof(ServeShared) + SERVE_RING * (sizeof(ServeReq) + sizeof(ServeDone)) + 256;
  if ((err = cudaHostAlloc(&h, bytes, cudaHostAllocMapped)) != cudaSuccess) {
    delete e;
    return berr(ctx, err, "serving rings");
  }
  std::memset(h, 0, bytes);
  void *hd = nullptr;
  if ((err = cudaHostGetDevicePointer(&hd, h, 0)) != cudaSuccess) {
    cudaFreeHost(h);
    delete e;
    return berr(ctx, err, "serving rings");
  }
  auto place = [&](size_t off, void **host, void **devp) {
    *host = static_cast<char *>(h) + off;
    *devp = static_cast<char *>(hd) + off;
  };
  const size_t o_req = (sizeof(ServeShared) + 127) & ~(size_t)127;
  const size_t o_done = o_req + SERVE_RING * sizeof(ServeReq);
  place(0, (void **)&e->sh, &e->sh_d);
  place(o_req, (void **)&e->reqs, &e->reqs_d);
  place(o_done, (void **)&e->dones, &e->dones_d);
  cudaEventCreateWithFlags(&e->done_ev, cudaEventDisableTiming);
  if ((rc = serve_reset_state(e))) {
    serve_engine_destroy(e);
    return rc;
  }
  serve_params(e);
  serve_capture(e);
  *out = e;
  return RPQ_OK;
}

void serve_engine_destroy(ServeEngine *e) {
  if (!e) return;
  if (e->running) cudaEventSynchronize(e->done_ev);
  cudaStreamSynchronize(ctx_stream(e->ctx));
  if (e->done_ev) cudaEventDestroy(e->done_ev);
  if (e->graph) cudaGraphExecDestroy(e->graph);
  if (e->sh) cudaFreeHost(e->sh);
  delete e;  // device buffers return to the context's budget
}

bool serve_engine_push(ServeEngine *e, uint64_t ticket, const QueryDesc &qd, uint32_t source) {
  const uint64_t tail = e->sh->req_tail;
  if (tail - e->sh->req_head >= SERVE_RING) return false;
  ServeReq *r = e->reqs + (tail & (SERVE_RING - 1));
  r->ticket = ticket;
  r->source = source;
  std::memcpy(&r->qd, &qd, sizeof(QueryDesc));
  std::atomic_thread_fence(std::memory_order_release);
  e->sh->req_tail = tail + 1;
  return true;
}

uint64_t serve_engine_waiting(ServeEngine *e) { return e->sh->req_tail - e->sh->req_head; }

void serve_engine_poll(ServeEngine *e, std::vector<ServeReply> *out) {
  const uint64_t tail = e->sh->done_tail;
  std::atomic_thread_fence(std::memory_order_acquire);
  uint64_t head = e->sh->done_head;
  for (; head < tail; head++) {
    const ServeDone &d = e->dones[head & (SERVE_RING - 1)];
    out->push_back({d.ticket, d.count, d.dsum, d.dxor, d.product_vertices, d.product_edges, d.evicted != 0});
  }
  std::atomic_thread_fence(std::memory_order_release);
  e->sh->done_head = head;
}

bool serve_engine_running(ServeEngine *e) {
  if (e->running && cudaEventQuery(e->done_ev) == cudaSuccess) e->running = false;
  return e->running;
}

void serve_engine_counters(ServeEngine *e, uint64_t *launches, uint64_t *admitted) {
  if (launches) *launches = e->launches;
  if (admitted) *admitted = e->sh->req_head;
}

int serve_engine_kick(ServeEngine *e, std::vector<uint64_t> *lost) {
  if (e->running) {
    const cudaError_t q = cudaEventQuery(e->done_ev);
    if (q == cudaErrorNotReady) return RPQ_OK;
    e->running = false;
    BfsCtl hctl;
    cudaError_t err = q;
    if (err == cudaSuccess) err = cudaMemcpy(&hctl, e->ctl.p, sizeof(BfsCtl), cudaMemcpyDeviceToHost);
    if (err != cudaSuccess) return berr(e->ctx, err, "serving launch");
    if (hctl.err) {
      // the launch stopped early: the requests in its slots are lost
      std::vector<u32> busy(e->slots);
      std::vector<u64> tk(e->slots);
      cudaMemcpy(busy.data(), e->busy.p, 4ull * e->slots, cudaMemcpyDeviceToHost);
      cudaMemcpy(tk.data(), e->tickets.p, 8ull * e->slots, cudaMemcpyDeviceToHost);
      for (uint32_t i = 0; i < e->slots; i++)
        if (busy[i]) lost->push_back(tk[i]);
      int rc = serve_reset_state(e);
      if (rc) return rc;
      if (hctl.err >= ERR_BOUNDS)
        return ctx_error(e->ctx, RPQ_ERR_CUDA, "serving launch index check " + std::to_string(hctl.err - ERR_BOUNDS));
      if (hctl.err == ERR_LIST_FULL) return ctx_error(e->ctx, RPQ_ERR_CUDA, "internal: serving list overflow");
      return ctx_error(e->ctx, RPQ_ERR_TIMEOUT, "serving launch grid barrier wait ran out of time");
    }
  }
  if (serve_engine_waiting(e) == 0) return RPQ_OK;
  cudaStream_t st = ctx_stream(e->ctx);
  cudaError_t err = e->graph ? cudaGraphLaunch(e->graph, st) : serve_issue(e, st);
  if (err == cudaSuccess) err = cudaEventRecord(e->done_ev, st);
  if (err != cudaSuccess) return berr(e->ctx, err, "serving launch");
  e->running = true;
  e->launches++;
  return RPQ_OK;
}

bool serve_engine_graphed(ServeEngine *e) { return e->graph != nullptr; }

int batch_run(rpq_ctx *ctx, const rpq_graph *g, uint32_t nq, const rpq_query *const *queries,
              const uint32_t *sources, bool materialize, const BatchTuning &tun, BatchOut *out) {
  const double t_start = host_seconds();
  if (out->per_query && !materialize && tun.direct && tun.lanes > 0) {
    // every query to the lane-mode launches
    out->qstats.assign(3ull * nq, 0);
    for (uint32_t i = 0; i < nq; i++) out->evicted_idx.push_back(i);
  }
  for (uint32_t b0 = 0; b0 < nq && out->evicted_idx.empty();) {
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
  out->qdone_ms.assign(nq, (host_seconds() - t_start) * 1e3);
  if (tun.lanes > 0) {
    // Queries that left the batch run with one lane each and their own
    // automaton in lane-mode launches of the multi-source engine.
    std::vector<LaneTask> tasks(out->evicted_idx.size());
    for (size_t j = 0; j < tasks.size(); j++) {
      tasks[j].q = queries[out->evicted_idx[j]];
      tasks[j].source = sources[out->evicted_idx[j]];
    }
    std::vector<uint64_t> ls;
    std::vector<double> done;
    rpq_stats st{};
    int rc = tasks.empty() ? RPQ_OK : rpq_lane_stats_lanes(ctx, g, tasks, tun.lanes, &ls, &st, &done);
    if (rc) return rc;
    for (size_t j = 0; j < tasks.size(); j++) {
      for (int c = 0; c < 3; c++) out->qstats[3ull * out->evicted_idx[j] + c] = ls[3 * j + c];
      out->qdone_ms[out->evicted_idx[j]] = (done[j] - t_start) * 1e3;
    }
    rpq_stats &a = out->stats;
    a.product_edges += st.product_edges;
    a.product_vertices += st.product_vertices;
    a.levels += st.levels;
    a.push_levels += st.push_levels;
    a.pull_levels += st.pull_levels;
    a.bfs_ms += st.bfs_ms;
    a.emit_ms += st.emit_ms;
    a.bfs_launches += st.bfs_launches;
    a.launches += st.launches;
    a.alg_bytes += st.alg_bytes;
    a.lane_groups += st.lane_groups;
    out->regroup_launches += st.bfs_launches;
  } else {
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
  for (uint32_t i : out->evicted_idx) out->qdone_ms[i] = (host_seconds() - t_start) * 1e3;
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
