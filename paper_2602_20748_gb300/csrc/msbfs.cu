// Product-graph breadth-first search for many start vertices at once.
//
// What is computed (Section 2.2, automata-based approach): for every start
// vertex s, the product vertices (v, q) of G x DFA reachable from (s, q0),
// with a visited set per start vertex so that each is expanded once; (s, v)
// is a result when some reached (v, q) has q accepting (Definition 1).  The
// search runs level by level until the frontier is empty, with no hop limit
// (the paper's Section 3 shows hop-limited depth-first search losing
// answers).
//
// How (design of this engine, not the paper's hop-limited DFS / segment
// pooling): start vertices are packed as bit lanes, K = 64 * NW of them per
// lane group, G groups per launch.  For every (state, vertex, group) there is
// one K-bit word in each of three arrays: VIS (visited) and two frontier
// words used in ping-pong, laid out [state][vertex][group][word] so that the
// G words of one (state, vertex) are contiguous (G * 8 * NW bytes, 512 for
// 16 groups of 256 lanes).  A level is expanded either
//   * top-down ("push"): the sparse list of (group, state, vertex) frontier
//     entries is scanned, the out-edges on the labels of the state's
//     transitions are spread evenly over the lanes of a warp, and the new
//     lanes are OR-ed into the next frontier word with atomics; rows longer
//     than SPILL_EDGES are cut into chunks shared by all warps; or
//   * bottom-up ("pull"): a warp takes one vertex and all groups at once: for
//     each in-edge on an incoming transition from a state that is present in
//     the frontier, it gathers the neighbour's G frontier words (one
//     coalesced 512-byte read) and ORs them into per-lane accumulators; rows
//     with at least HEAVY_ROW in-edges are cut (at graph load) into chunks
//     shared by all warps,
// chosen per level from the byte cost of each given the DFA states present
// in the frontier.  New lanes land in the next frontier word; a commit phase
// folds them into VIS and clears the old frontier.  The whole search is one
// persistent cooperative launch; levels are separated by a grid barrier whose
// waits are bounded by a time limit (on expiry the kernel records
// RPQ_ERR_TIMEOUT and returns).
#include "device_common.cuh"
#include "rpq_internal.h"

namespace rpq {

constexpr int BFS_THREADS = 256;

template <int NW>
struct Word {
  u64 w[NW];
};

template <int NW>
__device__ __forceinline__ Word<NW> load_cg(const u64 *p) {
  Word<NW> x;
  if constexpr (NW % 2 == 0) {
#pragma unroll
    for (int i = 0; i < NW; i += 2) {
      ulonglong2 a = __ldcg(reinterpret_cast<const ulonglong2 *>(p + i));
      x.w[i] = a.x;
      x.w[i + 1] = a.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < NW; i++) x.w[i] = __ldcg(p + i);
  }
  return x;
}

// PER consecutive words at p (16-byte aligned when PER is even), or all ones
// when !on.
template <int PER>
__device__ __forceinline__ void load_vis(const u64 *p, bool on, u64 (&v)[PER]) {
  if constexpr (PER % 2 == 0) {
#pragma unroll
    for (int k = 0; k < PER; k += 2) {
      const ulonglong2 a = on ? __ldcg(reinterpret_cast<const ulonglong2 *>(p + k)) : make_ulonglong2(~0ull, ~0ull);
      v[k] = a.x;
      v[k + 1] = a.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < PER; k++) v[k] = on ? __ldcg(p + k) : ~0ull;
  }
}

template <int NW>
__device__ __forceinline__ void store_w(u64 *p, const Word<NW> &x) {
  if constexpr (NW % 2 == 0) {
#pragma unroll
    for (int i = 0; i < NW; i += 2) *reinterpret_cast<ulonglong2 *>(p + i) = make_ulonglong2(x.w[i], x.w[i + 1]);
  } else {
#pragma unroll
    for (int i = 0; i < NW; i++) p[i] = x.w[i];
  }
}

template <int NW>
__device__ __forceinline__ bool any_bits(const Word<NW> &x) {
  u64 a = 0;
#pragma unroll
  for (int i = 0; i < NW; i++) a |= x.w[i];
  return a != 0;
}

template <int NW>
__device__ __forceinline__ u32 popc_w(const Word<NW> &x) {
  u32 c = 0;
#pragma unroll
  for (int i = 0; i < NW; i++) c += __popcll(x.w[i]);
  return c;
}

// First u64 of the word of (group g, state q, vertex v).
template <int NW>
__device__ __forceinline__ u64 widx(const BfsParams &p, u32 g, u32 q, u32 v) {
  return (((u64)q * p.n + v) * p.G + g) * NW;
}

// Grid-wide barrier for a cooperative launch.  Waits are bounded by the
// deadline; on expiry the error word is set and every block returns at its
// next check.  Returns false when the search must stop.
__device__ bool grid_barrier(BfsCtl *c, unsigned nblocks, u64 limit_ns) {
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
  // one reading per block, so all threads of a block take the same branch
  return stop == 0;
}

// Automaton modes of a launch: one automaton for every lane, one per lane
// group (multi), or one per lane (lane mode).
constexpr int AM_ONE = 0, AM_GROUP = 1, AM_LANE = 2;
// Lane-mode bottom-up by source state (see pull_level) for unions of at most
// this many states; larger ones gather per target state.
constexpr u32 LANE_SRC_Q = 8;

// Automaton of group g: its own in multi mode, else the launch's (the union
// in lane mode).
template <int AM>
__device__ __forceinline__ const QueryDesc &gdesc(const BfsParams &p, u32 g) {
  if constexpr (AM == AM_GROUP)
    return p.qg[g];
  else
    return p.q;
}

// Out-degree of v summed over the labels leaving DFA state q; *rows (if
// given) gets the number of those labels present in the graph.
__device__ __forceinline__ u32 degsum(const BfsParams &p, const QueryDesc &qd, u32 q, u32 v, u32 *rows = nullptr) {
  u32 s = 0, r = 0;
  const u32 n1 = p.n + 1;
  for (u32 t = qd.out_begin[q]; t < qd.out_begin[q + 1]; t++) {
    u32 l = qd.out_label[t];
    if (l >= p.L) continue;
    const u32 *off = p.out_off + (u64)l * n1 + v;
    s += __ldg(off + 1) - __ldg(off);
    r++;
  }
  if (rows) *rows = r;
  return s;
}

// Lane mode: the rows a top-down step over (q, v) reads -- the out-degree of
// v summed over the union's transitions leaving q (returned; their number in
// *rows) -- and, for the lanes set in m (group g's words), each lane's own
// product-edge count: deg_l(v) for every label l its automaton leaves q on,
// added into W.
template <int NW>
__device__ __forceinline__ u32 la_degsum(const BfsParams &p, u32 q, u32 v, u32 g, const Word<NW> &m, u64 &W,
                                         u32 *rows) {
  // per (state, label) group: its transitions' lanes are disjoint, so the
  // lanes of m taking any of them are popc(m & OR of their masks); the
  // degree sum and row count still count every transition
  u32 s = 0, r = 0;
  const u32 n1 = p.n + 1;
  const u64 gw = (u64)p.G * NW;
  for (u32 gi = p.la_grp_begin[q]; gi < p.la_grp_begin[q + 1]; gi++) {
    const u32 e = p.la_grp[gi];
    const u32 l = e & 0xFFFFu, c = e >> 16;
    if (l >= p.L) continue;
    const u32 *off = p.out_off + (u64)l * n1 + v;
    const u32 d = __ldg(off + 1) - __ldg(off);
    const u64 *mk = p.la_gmask + gi * gw + (u64)g * NW;
    u32 lanes = 0;
#pragma unroll
    for (int k = 0; k < NW; k++) lanes += __popcll(m.w[k] & __ldg(mk + k));
    W += (u64)lanes * d;
    s += c * d;
    r += c;
  }
  *rows = r;
  return s;
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

// A warp's current run of reserved list slots [pos, end) (warp-uniform).
struct Appender {
  u64 pos = 0, end = 0;
};

// Warp-aggregated append of `entry` for the lanes with `take` set.  All 32
// lanes must call it.  With segments, the warp fills its reserved slots and
// reserves APPEND_SEG more with one atomic add when they run out, so the
// list counter sees one atomic per segment instead of one per append.
__device__ __forceinline__ void warp_append(const BfsParams &p, Appender &a, bool take, u64 entry,
                                            unsigned long long *count, u64 *list) {
  const u32 b = __ballot_sync(FULL_MASK, take);
  if (!b) return;
  const u32 k = __popc(b), r = __popc(b & lanemask_lt());
  u64 at;
  if (p.append_seg == 0) {
    u64 base = 0;
    if (lane_id() == __ffs(b) - 1) base = atomicAdd(count, (unsigned long long)k);
    base = __shfl_sync(FULL_MASK, base, __ffs(b) - 1);
    at = base + r;
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
      atomicCAS(&p.ctl->err, 0u, ERR_LIST_OVERFLOW);
  }
}

// End of a phase: the warp's reserved slots not used hold NO_ENTRY.
__device__ __forceinline__ void append_close(const BfsParams &p, Appender &a, u64 *list) {
  for (u64 i = a.pos + lane_id(); i < a.end; i += 32)
    if (i < p.list_cap) list[i] = NO_ENTRY;
  a.pos = a.end = 0;
}

template <int NW, int AM>
__device__ void seed_phase(const BfsParams &p, u64 *stat) {
  const u32 K = 64 * NW;
  const u64 total = (u64)p.G * K;
  const u64 stride = (u64)gridDim.x * blockDim.x;
  u64 W = 0, N = 0, mf = 0, gx = 0, gn = 0;
  Appender app;
  for (u64 base = (u64)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < total; base += stride) {
    u64 i = base + lane_id();
    bool take = false;
    u64 entry = 0;
    if (i < total) {
      u32 s = p.lanesrc[i];
      if (s != NO_SOURCE) {
        u32 g = (u32)(i / K), lane = (u32)(i % K);
        u64 wi = widx<NW>(p, g, 0, s);  // start state 0
        // lanes may repeat a start vertex, so seeds share words: atomics, and
        // one list entry per (group, vertex)
        const u64 bit = 1ull << (lane % 64);
        atomicOr((unsigned long long *)(p.vis + wi + lane / 64), bit);
        const u64 oldf = atomicOr((unsigned long long *)(p.fr0 + wi + lane / 64), bit);
        if constexpr (NW == 1)
          take = oldf == 0;
        else
          take = atomicMax(p.claim + ((u64)s * p.G + g), p.stamp_base + 1) < p.stamp_base + 1;
        entry = ((u64)g * p.Q << 32) | s;
        if (take && p.fbits) atomicOr(p.fbits + (s >> 5), 1u << (s & 31));  // state 0, bitmap 0
        u32 rows = 0, d;
        if constexpr (AM == AM_LANE) {
          Word<NW> me;
#pragma unroll
          for (int k = 0; k < NW; k++) me.w[k] = (lane / 64 == (u32)k) ? bit : 0ull;
          d = la_degsum<NW>(p, 0, s, g, me, W, &rows);
        } else {
          d = degsum(p, gdesc<AM>(p, g), 0, s, &rows);
          W += d;
        }
        N += 1;
        if (take) {
          mf += d;
          gx += rows;
          gn += 1;
        }
      }
    }
    warp_append(p, app, take, entry, &p.ctl->n_list[0], p.list0);
  }
  append_close(p, app, p.list0);
  W = warp_sum(W);
  N = warp_sum(N);
  mf = warp_sum(mf);
  gx = warp_sum(gx);
  gn = warp_sum(gn);
  if (lane_id() == 0) {
    stat[ST_W] += W;
    stat[ST_N] += N;
    stat[ST_GROUP_VERTICES] += gn;
    // counted once per warp and phase: straight into the control block
    if (mf) atomicAdd(&p.ctl->stats[ST_GROUP_W], mf);
    if (gx) atomicAdd(&p.ctl->stats[ST_GROUP_X], gx);
    if (mf) atomicAdd(&p.ctl->mf[0], mf);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&p.ctl->smask[0], 1u);
}

// One top-down relaxation of edge (tgq, w) with source lanes fm: the lanes
// not yet visited at (tgq, w) are OR-ed into the next frontier word; returns
// whether this thread must list (tgq, w) in the next frontier.
template <int NW>
__device__ __forceinline__ bool relax(const BfsParams &p, u64 *FB, u32 tgq, u32 w, const Word<NW> &fm, u32 stamp) {
  const u32 g = tgq / p.Q, q2 = tgq - g * p.Q;
  const u64 wi = widx<NW>(p, g, q2, w);
  Word<NW> vis = load_cg<NW>(p.vis + wi);
  Word<NW> m;
#pragma unroll
  for (int i = 0; i < NW; i++) m.w[i] = fm.w[i] & ~vis.w[i];
  if (!any_bits(m)) return false;
  if constexpr (NW == 1) {
    u64 old = atomicOr((unsigned long long *)(FB + wi), m.w[0]);
    return old == 0;
  } else {
#pragma unroll
    for (int i = 0; i < NW; i++)
      if (m.w[i]) atomicOr((unsigned long long *)(FB + wi + i), m.w[i]);
    u32 old = atomicMax(p.claim + (((u64)q2 * p.n + w) * p.G + g), stamp);
    return old < stamp;
  }
}

// Top-down expansion of the entries of the current list.  A warp takes 32
// entries at a time and spreads the edges of their rows evenly over its lanes
// (prefix sum of row lengths, owner found by binary search); rows longer than
// SPILL_EDGES are queued in chunks for the spill sub-phase.
template <int NW, int AM>
__device__ void push_level(const BfsParams &p, int lp, u32 cur, u32 nxt, u64 n_cur, u32 stamp, u64 *stat) {
  const u64 *list = lp ? p.list1 : p.list0;
  u64 *nlist = lp ? p.list0 : p.list1;
  const u64 *F = lp ? p.fr1 : p.fr0;
  u64 *FB = lp ? p.fr0 : p.fr1;
  const u32 Q = p.Q, n1 = p.n + 1;
  const u32 lane = lane_id();
  u64 edges = 0, rows = 0, entries = 0;
  Appender app;
  for (;;) {
    u64 base = 0;
    if (lane == 0) base = atomicAdd(&p.ctl->cursor[cur], 32ull);
    base = __shfl_sync(FULL_MASK, base, 0);
    if (base >= n_cur) break;
    u64 idx = base + lane;
    u64 e = idx < n_cur ? __ldcg(&list[idx]) : NO_ENTRY;
    bool valid = e != NO_ENTRY;
    if (!valid) e = 0;
    u32 gq = (u32)(e >> 32), v = (u32)e;
    u32 g = gq / Q, q = gq - g * Q;
    Word<NW> fm;
#pragma unroll
    for (int i = 0; i < NW; i++) fm.w[i] = 0;
    if (valid) fm = load_cg<NW>(F + widx<NW>(p, g, q, v));
    entries += valid;
    const QueryDesc &qd = gdesc<AM>(p, valid ? g : 0);
    u32 t_beg, nt;
    if constexpr (AM == AM_LANE) {
      t_beg = valid ? p.la_out_begin[q] : 0;
      nt = valid ? p.la_out_begin[q + 1] - t_beg : 0;
    } else {
      t_beg = valid ? qd.out_begin[q] : 0;
      nt = valid ? qd.out_begin[q + 1] - t_beg : 0;
    }
    u32 max_nt = __reduce_max_sync(FULL_MASK, nt);
    for (u32 j = 0; j < max_nt; j++) {
      u32 rbeg = 0, rlen = 0, tgq = 0;
      Word<NW> fmt = fm;  // the entry's lanes that take this transition
      if (j < nt) {
        u32 t = t_beg + j;
        u32 l, to;
        if constexpr (AM == AM_LANE) {
          const u32 e = p.la_trans[t];
          l = e & 0xFFFFu;
          to = e >> 16;
          const u64 *mk = p.la_mask + (u64)t * ((u64)p.G * NW) + (u64)g * NW;
#pragma unroll
          for (int k = 0; k < NW; k++) fmt.w[k] &= __ldg(mk + k);
        } else {
          l = qd.out_label[t];
          to = qd.out_to[t];
        }
        tgq = g * Q + to;
        if (l < p.L && (AM != AM_LANE || any_bits(fmt))) {
          const u32 *off = p.out_off + (u64)l * n1 + v;
          rbeg = __ldg(off);
          rlen = __ldg(off + 1) - rbeg;
          rows++;
        }
      }
      if (p.spill && rlen > SPILL_EDGES) {
        const u32 chunks = (rlen + SPILL_EDGES - 1) / SPILL_EDGES;
        u64 at = 0;
        const u32 fit = spill_reserve(&p.ctl->spill_count[cur], chunks, p.spill_cap, &at);
        for (u32 c = 0; c < fit; c++) {
          u64 *rec = p.spill + (at + c) * (2 + NW);
          rec[0] = ((u64)tgq << 32) | (rbeg + c * SPILL_EDGES);
          rec[1] = min(SPILL_EDGES, rlen - c * SPILL_EDGES);
#pragma unroll
          for (int t = 0; t < NW; t++) rec[2 + t] = fmt.w[t];
        }
        // the chunks that did not fit stay with this warp
        const u32 moved = min(rlen, fit * SPILL_EDGES);
        rbeg += moved;
        rlen -= moved;
      }
      // exclusive prefix of row lengths across the warp
      u32 pre = rlen;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        u32 t = __shfl_up_sync(FULL_MASK, pre, o);
        if (lane >= (u32)o) pre += t;
      }
      u32 total = __shfl_sync(FULL_MASK, pre, 31);
      pre -= rlen;
      edges += (lane == 0) ? total : 0;
      for (u32 k0 = 0; k0 < total; k0 += 32) {
        u32 k = k0 + lane;
        // owner: the largest lane o with pre[o] <= k
        u32 o = 0;
#pragma unroll
        for (u32 step = 16; step > 0; step >>= 1) {
          u32 pv = __shfl_sync(FULL_MASK, pre, o + step);
          if (pv <= k) o += step;
        }
        u32 o_beg = __shfl_sync(FULL_MASK, rbeg, o);
        u32 o_pre = __shfl_sync(FULL_MASK, pre, o);
        u32 o_gq = __shfl_sync(FULL_MASK, tgq, o);
        Word<NW> ofm;
#pragma unroll
        for (int i = 0; i < NW; i++) ofm.w[i] = __shfl_sync(FULL_MASK, fmt.w[i], o);
        bool take = false;
        u32 w = 0;
        if (k < total) {
          w = __ldg(p.out_col + o_beg + (k - o_pre));
          take = relax<NW>(p, FB, o_gq, w, ofm, stamp);
        }
        warp_append(p, app, take, ((u64)o_gq << 32) | w, &p.ctl->n_list[nxt], nlist);
      }
    }
  }
  append_close(p, app, nlist);
  edges = warp_sum(edges);
  rows = warp_sum(rows);
  entries = warp_sum(entries);
  stat[ST_GROUP_EDGES] += edges;
  stat[ST_GROUP_ROWS] += rows;
  // per relaxation a column id and the target's visited word (the spilled
  // share is counted by the spill phase); per row its two offsets; per entry
  // the list entry and its frontier word
  stat[ST_ALG_BYTES] += edges * (4 + 8 * NW) + rows * 8 + entries * (8 + 8 * NW);
}

// The queued chunks of long rows: a warp per chunk, taken dynamically.
template <int NW>
__device__ void spill_phase(const BfsParams &p, int lp, u32 cur, u32 nxt, u32 stamp, u64 *stat) {
  u64 *nlist = lp ? p.list0 : p.list1;
  u64 *FB = lp ? p.fr0 : p.fr1;
  const u32 lane = lane_id();
  const u64 count = min(*(volatile unsigned long long *)&p.ctl->spill_count[cur], (unsigned long long)p.spill_cap);
  u64 edges = 0;
  Appender app;
  for (;;) {
    u64 r = 0;
    if (lane == 0) r = atomicAdd(&p.ctl->spill_cursor[cur], 1ull);
    r = __shfl_sync(FULL_MASK, r, 0);
    if (r >= count) break;
    const u64 *rec = p.spill + r * (2 + NW);
    const u64 h = __ldcg(rec);
    const u32 tgq = (u32)(h >> 32), b = (u32)h;
    const u32 len = (u32)__ldcg(rec + 1);
    Word<NW> fm;
#pragma unroll
    for (int t = 0; t < NW; t++) fm.w[t] = __ldcg(rec + 2 + t);
    edges += (lane == 0) ? len : 0;
    for (u32 k0 = 0; k0 < len; k0 += 32) {
      u32 k = k0 + lane;
      bool take = false;
      u32 w = 0;
      if (k < len) {
        w = __ldg(p.out_col + b + k);
        take = relax<NW>(p, FB, tgq, w, fm, stamp);
      }
      warp_append(p, app, take, ((u64)tgq << 32) | w, &p.ctl->n_list[nxt], nlist);
    }
  }
  append_close(p, app, nlist);
  edges = warp_sum(edges);
  stat[ST_GROUP_EDGES] += edges;
  stat[ST_ALG_BYTES] += edges * (4 + 8 * NW);
}

// Bottom-up work for target (q2, w) over in-edges [beg, end) of one
// transition group with active source states `from`: every lane ORs the
// gathered frontier words of its PER words into acc.  With EARLY (one lane
// group: few enough lanes that a vertex can run out of unvisited ones) a lane
// stops gathering once acc covers all its lanes not yet visited, and the
// sub-warp (lanes sg_mask) leaves the row when all its lanes have (with many
// groups a vertex practically never runs out, and the test costs more than it
// saves).  Returns the in-edges examined.
template <int NW, int PER, bool EARLY, bool LANE>
__device__ __forceinline__ u32 gather_row(const BfsParams &p, const u64 *F, const u32 *bits, u32 from, u32 beg,
                                          u32 end, u32 lane_off, bool lane_on, u32 sg_mask,
                                          const u64 (&vis)[PER], u64 (&acc)[PER], u32 &gathers,
                                          const unsigned short *tin) {
  const u32 n = p.n;
  const u64 wpv = (u64)p.G * NW;
  // lane mode: the gathered words of source state s are masked with the lanes
  // that take this group's transition from s (tin[s]); else all lanes
  auto lane_mask = [&](u32 st, u64 (&mk)[PER]) {
    if constexpr (LANE) {
      const u64 *mp = p.la_mask + (u64)tin[st] * wpv + lane_off;
#pragma unroll
      for (int k = 0; k < PER; k++) mk[k] = __ldg(mp + k);
    } else {
#pragma unroll
      for (int k = 0; k < PER; k++) mk[k] = ~0ull;
    }
  };
  auto done = [&]() {
    bool d = true;
#pragma unroll
    for (int k = 0; k < PER; k++) d &= (acc[k] | vis[k]) == ~0ull;
    return d;
  };
  // a lane with no source state on this row (another group's label in a
  // multi launch) has nothing to gather here
  bool fin = !lane_on || from == 0 || (EARLY && done());
  if (EARLY && (__ballot_sync(sg_mask, !fin) & sg_mask) == 0) return 0;
  u32 i = beg;
  // four in-edges per step keep four gathers in flight
  for (; i + 4 <= end; i += 4) {
    u32 v0 = __ldg(p.in_col + i), v1 = __ldg(p.in_col + i + 1), v2 = __ldg(p.in_col + i + 2),
        v3 = __ldg(p.in_col + i + 3);
    if (!fin) {
      for (u32 fb = from; fb; fb &= fb - 1) {
        u64 mk[PER];
        lane_mask(__ffs(fb) - 1, mk);
        const u64 qb = (u64)(__ffs(fb) - 1) * n;
        // with a frontier bitmap, neighbours outside the frontier are skipped
        bool h0 = true, h1 = true, h2 = true, h3 = true;
        if (bits) {
          h0 = (__ldcg(bits + ((qb + v0) >> 5)) >> ((qb + v0) & 31)) & 1u;
          h1 = (__ldcg(bits + ((qb + v1) >> 5)) >> ((qb + v1) & 31)) & 1u;
          h2 = (__ldcg(bits + ((qb + v2) >> 5)) >> ((qb + v2) & 31)) & 1u;
          h3 = (__ldcg(bits + ((qb + v3) >> 5)) >> ((qb + v3) & 31)) & 1u;
        }
        gathers += (u32)h0 + (u32)h1 + (u32)h2 + (u32)h3;
        const u64 *f0 = F + (qb + v0) * wpv + lane_off, *f1 = F + (qb + v1) * wpv + lane_off;
        const u64 *f2 = F + (qb + v2) * wpv + lane_off, *f3 = F + (qb + v3) * wpv + lane_off;
        if constexpr (PER == 2) {
          const ulonglong2 z = make_ulonglong2(0, 0);
          ulonglong2 a0 = h0 ? __ldcg(reinterpret_cast<const ulonglong2 *>(f0)) : z;
          ulonglong2 a1 = h1 ? __ldcg(reinterpret_cast<const ulonglong2 *>(f1)) : z;
          ulonglong2 a2 = h2 ? __ldcg(reinterpret_cast<const ulonglong2 *>(f2)) : z;
          ulonglong2 a3 = h3 ? __ldcg(reinterpret_cast<const ulonglong2 *>(f3)) : z;
          acc[0] |= (a0.x | a1.x | a2.x | a3.x) & mk[0];
          acc[1] |= (a0.y | a1.y | a2.y | a3.y) & mk[1];
        } else {
          acc[0] |= ((h0 ? __ldcg(f0) : 0ull) | (h1 ? __ldcg(f1) : 0ull) | (h2 ? __ldcg(f2) : 0ull) |
                     (h3 ? __ldcg(f3) : 0ull)) &
                    mk[0];
        }
      }
      if (EARLY) fin = done();
    }
    if (EARLY && (__ballot_sync(sg_mask, !fin) & sg_mask) == 0) return i + 4 - beg;
  }
  for (; i < end; i++) {
    u32 v = __ldg(p.in_col + i);
    if (fin) continue;
    for (u32 fb = from; fb; fb &= fb - 1) {
      const u64 bi = (u64)(__ffs(fb) - 1) * n + v;
      if (bits && !((__ldcg(bits + (bi >> 5)) >> (bi & 31)) & 1u)) continue;
      gathers++;
      u64 mk[PER];
      lane_mask(__ffs(fb) - 1, mk);
      const u64 *f = F + bi * wpv + lane_off;
#pragma unroll
      for (int k = 0; k < PER; k++) acc[k] |= __ldcg(f + k) & mk[k];
    }
  }
  return end - beg;
}

// Bottom-up target (q2, w), all groups: new lanes = acc & ~VIS go to the next
// frontier word, and one lane per group appends the list entry.  When chunks
// of long in-rows of the same vertex may also produce (q2, w) in this level
// (shared), the word is or-ed atomically and the entry is claimed (the first
// producer appends); otherwise this sub-warp is the only producer, the word
// was zero, and no atomic result has to be waited for.
template <int NW, int PER>
__device__ __forceinline__ void pull_finish(const BfsParams &p, Appender &app, u64 *FB, u64 *nlist, u32 nxt, u32 q2,
                                            u32 w, u32 stamp, u32 lane, bool lane_on, u32 my_g, bool shared,
                                            const u64 (&vis)[PER], const u64 (&acc)[PER]) {
  const u64 base = ((u64)q2 * p.n + w) * p.G * NW + (u64)lane * PER;
  bool take = false;
  bool nz = false;
  u64 nw[PER];
#pragma unroll
  for (int k = 0; k < PER; k++) {
    nw[k] = lane_on ? (acc[k] & ~vis[k]) : 0;
    nz |= nw[k] != 0;
  }
  if constexpr (NW == 1) {
    if (nz) {
      if (shared) {
        take = atomicOr((unsigned long long *)(FB + base), nw[0]) == 0;
      } else {
        FB[base] = nw[0];
        take = true;
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < PER; k++)
      if (nw[k]) {
        if (shared)
          atomicOr((unsigned long long *)(FB + base + k), nw[k]);
        else
          FB[base + k] = nw[k];
      }
    // NW / PER lanes hold one group's word
    bool gnz = nz;
#pragma unroll
    for (int o = 1; o < NW / PER; o <<= 1) gnz |= __shfl_xor_sync(FULL_MASK, gnz, o);
    if (gnz && lane_on && (lane % (NW / PER)) == 0)
      take = !shared || atomicMax(p.claim + (((u64)q2 * p.n + w) * p.G + my_g), stamp) < stamp;
  }
  warp_append(p, app, take, ((u64)(my_g * p.Q + q2) << 32) | w, &p.ctl->n_list[nxt], nlist);
}

// Bottom-up expansion.  Light rows: one vertex per sub-warp of SW lanes (the
// smallest power of two holding the vertex's G * NW words at PER words per
// lane), all groups at once, so a warp covers 32 / SW vertices (32 for a
// single start vertex).  Long rows: their precomputed chunks, a warp per
// chunk taken dynamically over the (target state, transition group) pairs
// whose source states are active; the sub-warps split the chunk's edges and
// OR their gathers together.
template <int NW, bool EARLY, int AM>
__device__ void pull_level(const BfsParams &p, int lp, u32 cur, u32 nxt, u32 active, u32 stamp, const u32 *bits,
                           u64 *stat) {
  constexpr int PER = (NW >= 2) ? 2 : 1;
  const u64 *F = lp ? p.fr1 : p.fr0;
  u64 *FB = lp ? p.fr0 : p.fr1;
  u64 *nlist = lp ? p.list0 : p.list1;
  const u32 n = p.n, Q = p.Q, n1 = p.n + 1;
  const u32 lane = lane_id();
  const u32 lanes_used = p.G * NW / PER;
  u32 SW = 1;
  while (SW < lanes_used) SW <<= 1;
  const u32 VPW = 32 / SW;  // vertices per warp
  const u32 sg = lane / SW, li = lane % SW;
  const u32 sg_mask = SW == 32 ? FULL_MASK : (((1u << SW) - 1u) << (sg * SW));
  const bool lane_on = li < lanes_used;
  const u32 lane_off = li * PER;
  const u32 my_g = lane_on ? lane_off / NW : 0;
  const u64 wpv = (u64)p.G * NW;
  const u64 warp = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const u64 n_warps = ((u64)gridDim.x * blockDim.x) >> 5;
  const bool chunked = p.hchunk != nullptr;
  const u64 gword = 8ull * NW * p.G;  // bytes of the G words of one (state, vertex)
  u64 edges = 0, words = 0, bytes = 0;
  Appender app;
  // lane mode by source state: this warp's per-target accumulators
  u64 *lane_acc = nullptr;
  if constexpr (AM == AM_LANE) {
    __shared__ u64 s_lane_acc[BFS_THREADS / 32][LANE_SRC_Q * 2 * 32];
    lane_acc = s_lane_acc[threadIdx.x >> 5];
  }

  // A warp takes 32 consecutive vertices at a time: lane i first finds, with
  // coalesced reads of the in-row offsets, the target states into which
  // vertex c0 + i has a light in-row on an active transition; only those
  // (vertex, state) pairs are then visited, VPW vertices at a time (their
  // offsets are in L1 by then).  With pull_dynamic the chunks are taken from
  // a cursor (the level's list cursor, unused by bottom-up levels), so a
  // warp whose chunks had little work takes more of them; else chunk k goes
  // to warp k mod warps.
  u64 c0 = warp * 32;
  if (p.pull_dynamic) {
    u64 t = 0;
    if (lane == 0) t = atomicAdd(&p.ctl->cursor[cur], 32ull);
    c0 = __shfl_sync(FULL_MASK, t, 0);
  }
  for (; c0 < n;) {
    // hmask: states with a long in-row (its chunks also produce); with a
    // sparse frontier (bits), lane i also tests up to PRESCAN in-edges of
    // its own vertex against the frontier bitmap, so that a state none of
    // whose in-neighbours is in the frontier is dropped here, 32 vertices at
    // a time; tmask: states whose light rows are longer than that and showed
    // no hit yet -- the sub-warp tests the rest of them below
    constexpr u32 PRESCAN = 16;
    u32 qmask = 0, hmask = 0, tmask = 0;
    if (c0 + lane < n) {
      const u32 v = (u32)(c0 + lane);
      for (u32 q2 = 0; q2 < Q; q2++)
        for (u32 j = p.q.in_begin[q2]; j < p.q.in_begin[q2 + 1]; j++) {
          const u32 l = p.q.in_label[j];
          const u32 from = p.q.in_from[j] & active;
          if (!from || l >= p.L) continue;
          const u32 *off = p.in_off + (u64)l * n1 + v;
          const u32 beg = __ldg(off), len = __ldg(off + 1) - beg;
          if (len >= HEAVY_ROW && chunked) {
            hmask |= 1u << q2;
            continue;
          }
          if (len == 0 || (((qmask & ~tmask) >> q2) & 1u)) continue;  // a hit is known already
          if (!bits) {
            qmask |= 1u << q2;
            continue;
          }
          bool hit = false;
          const u32 scan = min(len, PRESCAN);
          for (u32 i = 0; i < scan && !hit; i += 4) {
            u32 u[4];
#pragma unroll
            for (int t = 0; t < 4; t++) u[t] = i + t < scan ? __ldg(p.in_col + beg + i + t) : NO_SOURCE;
            for (u32 fb = from; fb; fb &= fb - 1) {
              const u64 qb = (u64)(__ffs(fb) - 1) * n;
#pragma unroll
              for (int t = 0; t < 4; t++)
                if (u[t] != NO_SOURCE) hit |= (__ldcg(bits + ((qb + u[t]) >> 5)) >> ((qb + u[t]) & 31)) & 1u;
            }
          }
          bytes += (u64)scan * (4 + 4 * __popc(from));
          if (hit) {
            qmask |= 1u << q2;
            tmask &= ~(1u << q2);
          } else if (len > PRESCAN) {
            qmask |= 1u << q2;
            tmask |= 1u << q2;
          }
        }
    }
    const u32 M = __ballot_sync(FULL_MASK, qmask != 0);
    for (u32 s0 = 0; s0 < 32 && (M >> s0); s0 += VPW) {
      if (VPW < 32 && ((M >> s0) & ((1u << VPW) - 1u)) == 0) continue;
      const u32 s = s0 + sg;
      const u32 vq = __shfl_sync(FULL_MASK, qmask, s);
      const u32 vh = __shfl_sync(FULL_MASK, hmask, s);
      const u32 vt = __shfl_sync(FULL_MASK, tmask, s);
      const bool wv = vq != 0;
      const u32 w = wv ? (u32)(c0 + s) : 0;
    if constexpr (AM == AM_LANE) {
      if (p.lane_by_source && Q <= LANE_SRC_Q) {
        // Lane mode by source state.  Target q2's new lanes are the OR over
        // its union transitions t = (s, l, q2) and the in-edges (v, w) of
        // label l of F[s][v] & mask(t); since the mask does not depend on v,
        // that is the OR over t of mask(t) & (OR over v of F[s][v]).  So the
        // frontier words of each (label, source state) are gathered once and
        // ORed over the in-edges, then masked into every target taking a
        // transition from them (accumulated per lane in shared memory); the
        // per-target order gathers each (s, v) once per target instead.
        u64 *sacc = lane_acc;  // [q2][k][lane]
        u32 wmask = 0;  // targets with lanes to find (uniform within the sub-warp)
        for (u32 q2 = 0; q2 < Q; q2++) {
          const bool any = wv && ((vq >> q2) & 1u);
          u64 vis[PER];
          load_vis<PER>(p.vis + ((u64)q2 * n + w) * wpv + lane_off, lane_on && any, vis);
          bool full = true;
#pragma unroll
          for (int k = 0; k < PER; k++) {
            full &= vis[k] == ~0ull;
            sacc[(q2 * PER + k) * 32 + lane] = 0;
          }
          const u32 fb = __ballot_sync(FULL_MASK, full);
          if (any && (fb & sg_mask) != sg_mask) wmask |= 1u << q2;
        }
        u64 lset = 0;  // labels of the work targets' active transitions
        for (u32 q2 = 0; q2 < Q; q2++)
          if ((wmask >> q2) & 1u)
            for (u32 j = p.q.in_begin[q2]; j < p.q.in_begin[q2 + 1]; j++)
              if ((p.q.in_from[j] & active) && p.q.in_label[j] < p.L) lset |= 1ull << p.q.in_label[j];
        for (; lset; lset &= lset - 1) {
          const u32 l = __ffsll((long long)lset) - 1;
          const u32 *off = p.in_off + (u64)l * n1 + w;
          const u32 beg = __ldg(off), end = __ldg(off + 1);
          if (beg == end || (end - beg >= HEAVY_ROW && chunked)) continue;
          u32 S = 0;  // source states of those transitions on label l
          for (u32 q2 = 0; q2 < Q; q2++)
            if ((wmask >> q2) & 1u)
              for (u32 j = p.q.in_begin[q2]; j < p.q.in_begin[q2 + 1]; j++)
                if (p.q.in_label[j] == l) S |= p.q.in_from[j] & active;
          for (; S; S &= S - 1) {
            const u32 st = __ffs(S) - 1;
            u64 g[PER], none[PER];
#pragma unroll
            for (int k = 0; k < PER; k++) g[k] = none[k] = 0;
            u32 gat = 0;
            const u32 ex = gather_row<NW, PER, false, false>(p, F, bits, 1u << st, beg, end, lane_off, lane_on,
                                                             sg_mask, none, g, gat, nullptr);
            edges += (li == 0) ? ex : 0;
            bytes += (li == 0) ? 8 + (u64)ex * (4 + (bits ? 4 : 0)) + (u64)gat * gword : 0;
            bool nz = false;
#pragma unroll
            for (int k = 0; k < PER; k++) nz |= g[k] != 0;
            if (!nz) continue;
            for (u32 q2 = 0; q2 < Q; q2++) {
              if (!((wmask >> q2) & 1u)) continue;
              for (u32 j = p.q.in_begin[q2]; j < p.q.in_begin[q2 + 1]; j++) {
                if (p.q.in_label[j] != l || !((p.q.in_from[j] >> st) & 1u)) continue;
                const u64 *mk = p.la_mask + (u64)p.la_in_t[(u64)j * Q + st] * wpv + lane_off;
#pragma unroll
                for (int k = 0; k < PER; k++) sacc[(q2 * PER + k) * 32 + lane] |= g[k] & __ldg(mk + k);
              }
            }
          }
        }
        for (u32 q2 = 0; q2 < Q; q2++) {
          const bool work = ((wmask >> q2) & 1u) != 0;
          if (!__any_sync(FULL_MASK, work)) continue;
          u64 vis[PER], acc[PER];
          load_vis<PER>(p.vis + ((u64)q2 * n + w) * wpv + lane_off, lane_on && work, vis);
#pragma unroll
          for (int k = 0; k < PER; k++) acc[k] = sacc[(q2 * PER + k) * 32 + lane];
          words += (li == 0 && work);
          bytes += (li == 0 && work) ? gword : 0;
          pull_finish<NW, PER>(p, app, FB, nlist, nxt, q2, w, stamp, li, lane_on && work, my_g,
                               ((vh >> q2) & 1u) != 0, vis, acc);
        }
        continue;
      }
    }
    for (u32 q2 = 0; q2 < Q; q2++) {
      const u32 gb = p.q.in_begin[q2], ge = p.q.in_begin[q2 + 1];
      bool any = wv && ((vq >> q2) & 1u);
      if (bits && __any_sync(FULL_MASK, any && ((vt >> q2) & 1u))) {
        // sparse frontier, rows the pre-scan left undecided: a vertex none of
        // whose in-neighbours is in the frontier is skipped before its
        // visited words are read (the sub-warp's lanes test the in-edges in
        // turn: a column id and a bitmap word each)
        bool hit = false;
        if (!((vt >> q2) & 1u)) any = false, hit = wv && ((vq >> q2) & 1u);
        for (u32 j = gb; j < ge && !hit && any; j++) {
          const u32 l = p.q.in_label[j];
          const u32 from = p.q.in_from[j] & active;
          if (!from || l >= p.L) continue;
          const u32 *off = p.in_off + (u64)l * n1 + w;
          const u32 beg = __ldg(off), end = __ldg(off + 1);
          if (end - beg >= HEAVY_ROW && chunked) continue;
          for (u32 i = beg + li; i < end && !hit; i += SW) {
            const u32 u = __ldg(p.in_col + i);
            bytes += 4 + 4 * __popc(from);
            for (u32 fb = from; fb && !hit; fb &= fb - 1) {
              const u64 bi = (u64)(__ffs(fb) - 1) * n + u;
              hit = (__ldcg(bits + (bi >> 5)) >> (bi & 31)) & 1u;
            }
          }
        }
        any = (__ballot_sync(FULL_MASK, hit) & sg_mask) != 0;
      }
      const u64 base = ((u64)q2 * n + w) * wpv + lane_off;
      u64 vis[PER];
      load_vis<PER>(p.vis + base, lane_on && any, vis);
      u64 acc[PER];
#pragma unroll
      for (int k = 0; k < PER; k++) acc[k] = 0;
      // the in-rows' gathers into acc
      auto gather_all = [&]() {
        for (u32 j = gb; j < ge; j++) {
          const u32 l = p.q.in_label[j];
          const u32 from = p.q.in_from[j] & active;
          if (!from || l >= p.L) continue;
          const u32 *off = p.in_off + (u64)l * n1 + w;
          const u32 beg = __ldg(off), end = __ldg(off + 1);
          if (end - beg >= HEAVY_ROW && chunked) continue;
          // in multi mode each lane gathers through its own group's transitions
          u32 lfrom = from;
          if constexpr (AM == AM_GROUP) lfrom = lane_on ? p.from_tab[((u64)my_g * Q + q2) * p.L + l] & active : 0u;
          u32 gat = 0;
          const u32 ex = gather_row<NW, PER, EARLY, AM == AM_LANE>(p, F, bits, lfrom, beg, end, lane_off, lane_on,
                                                                   sg_mask, vis, acc, gat,
                                                                   p.la_in_t + (u64)j * Q);
          edges += (li == 0) ? ex : 0;
          // column ids, frontier-bit words when tested, gathered frontier words
          bytes += (li == 0) ? 8 + (u64)ex * (4 + (bits ? 4 * __popc(from) : 0)) + (u64)gat * gword : 0;
        }
        words += (li == 0);
        bytes += (li == 0) ? gword : 0;
      };
      // whether every lane of the sub-warp's vertex is visited; a warp-wide
      // ballot, so every lane of the warp must call it
      auto all_visited = [&]() {
        bool full = true;
#pragma unroll
        for (int k = 0; k < PER; k++) full &= vis[k] == ~0ull;
        return (__ballot_sync(FULL_MASK, full) & sg_mask) == sg_mask;
      };
      bool work;
      if constexpr (EARLY) {
        // the gathers stop early on the visited words: read them first
        const bool allv = all_visited();
        work = any && !allv;
        if (!__any_sync(FULL_MASK, work)) continue;
        if (work) gather_all();
      } else {
        // the gathers do not read the visited words, so they are issued while
        // those are in flight (a vertex whose lanes turn out all visited
        // gathered for nothing: rare where many lanes never reach anything)
        if (!__any_sync(FULL_MASK, any)) continue;
        if (any) gather_all();
        const bool allv = all_visited();
        work = any && !allv;
        if (!__any_sync(FULL_MASK, work)) continue;
      }
      pull_finish<NW, PER>(p, app, FB, nlist, nxt, q2, w, stamp, li, lane_on && work, my_g, ((vh >> q2) & 1u) != 0,
                           vis, acc);
    }
    }
    if (p.pull_dynamic) {
      u64 t = 0;
      if (lane == 0) t = atomicAdd(&p.ctl->cursor[cur], 32ull);
      c0 = __shfl_sync(FULL_MASK, t, 0);
    } else {
      c0 += n_warps * 32;
    }
  }

  bool chunks_done = !chunked;
  if constexpr (AM == AM_LANE) {
    if (chunked && p.lane_by_source && Q <= LANE_SRC_Q) {
      // Long in-rows by source state: an item is a chunk of a label's long
      // in-rows; its frontier words are gathered once per active source
      // state with a transition on that label and masked into every target
      // taking one (the light rows' scheme, see above).
      u64 lact = 0;  // labels with an active transition
      for (u32 j = 0; j < p.q.in_begin[Q]; j++)
        if ((p.q.in_from[j] & active) && p.q.in_label[j] < p.L) lact |= 1ull << p.q.in_label[j];
      for (;;) {
        u64 it = 0;
        if (lane == 0) it = atomicAdd(&p.ctl->heavy_cursor[cur], 1ull);
        it = __shfl_sync(FULL_MASK, it, 0);
        u64 acc_base = 0, ci = 0;
        u32 ls = 0;
        bool found = false;
        for (u64 lb = lact; lb; lb &= lb - 1) {
          const u32 l = __ffsll((long long)lb) - 1;
          const u64 cnt = p.hchunk_off[l + 1] - p.hchunk_off[l];
          if (it < acc_base + cnt) {
            found = true;
            ls = l;
            ci = p.hchunk_off[l] + (it - acc_base);
            break;
          }
          acc_base += cnt;
        }
        if (!found) break;
        const u32 *rec = p.hchunk + 3 * ci;
        const u32 w = __ldg(rec), beg = __ldg(rec + 1), end = __ldg(rec + 2);
        // targets with a transition on ls from an active state and lanes not
        // yet visited (the whole warp works on vertex w)
        u32 wmask = 0;
        for (u32 q2 = 0; q2 < Q; q2++) {
          bool has = false;
          for (u32 j = p.q.in_begin[q2]; j < p.q.in_begin[q2 + 1]; j++)
            has |= p.q.in_label[j] == ls && (p.q.in_from[j] & active) != 0;
          u64 vis[PER];
          load_vis<PER>(p.vis + ((u64)q2 * n + w) * wpv + lane_off, lane_on && has, vis);
          bool full = true;
#pragma unroll
          for (int k = 0; k < PER; k++) {
            full &= vis[k] == ~0ull;
            lane_acc[(q2 * PER + k) * 32 + lane] = 0;
          }
          const u32 fbal = __ballot_sync(FULL_MASK, full);  // every lane, before the test
          if (has && fbal != FULL_MASK) wmask |= 1u << q2;
        }
        if (!wmask) continue;
        u32 S = 0;
        for (u32 q2 = 0; q2 < Q; q2++)
          if ((wmask >> q2) & 1u)
            for (u32 j = p.q.in_begin[q2]; j < p.q.in_begin[q2 + 1]; j++)
              if (p.q.in_label[j] == ls) S |= p.q.in_from[j] & active;
        // the sub-warps take consecutive slices of the chunk's edges
        const u32 len = end - beg, per = (len + VPW - 1) / VPW;
        const u32 sb = beg + min(len, sg * per), se = beg + min(len, (sg + 1) * per);
        u64 ex_tot = 0, gat_tot = 0;
        for (; S; S &= S - 1) {
          const u32 st = __ffs(S) - 1;
          u64 g[PER], none[PER];
#pragma unroll
          for (int k = 0; k < PER; k++) g[k] = none[k] = 0;
          u32 gat = 0;
          ex_tot += gather_row<NW, PER, false, false>(p, F, bits, 1u << st, sb, se, lane_off, lane_on, sg_mask,
                                                      none, g, gat, nullptr);
          gat_tot += gat;
          for (u32 o = SW; o < 32; o <<= 1) {
#pragma unroll
            for (int k = 0; k < PER; k++) g[k] |= __shfl_xor_sync(FULL_MASK, g[k], o);
          }
          for (u32 q2 = 0; q2 < Q; q2++) {
            if (!((wmask >> q2) & 1u)) continue;
            for (u32 j = p.q.in_begin[q2]; j < p.q.in_begin[q2 + 1]; j++) {
              if (p.q.in_label[j] != ls || !((p.q.in_from[j] >> st) & 1u)) continue;
              const u64 *mk = p.la_mask + (u64)p.la_in_t[(u64)j * Q + st] * wpv + lane_off;
#pragma unroll
              for (int k = 0; k < PER; k++) lane_acc[(q2 * PER + k) * 32 + lane] |= g[k] & __ldg(mk + k);
            }
          }
        }
        const u64 ex_all = warp_sum((u64)(li == 0 ? ex_tot : 0));
        const u64 gat_all = warp_sum((u64)(li == 0 ? gat_tot : 0));
        edges += (lane == 0) ? ex_all : 0;
        bytes += (lane == 0) ? 12 + ex_all * (4 + (bits ? 4 : 0)) + gat_all * gword : 0;
        for (u32 q2 = 0; q2 < Q; q2++) {
          if (!((wmask >> q2) & 1u)) continue;  // uniform across the warp
          u64 vis[PER], acc[PER];
          load_vis<PER>(p.vis + ((u64)q2 * n + w) * wpv + lane_off, lane_on, vis);
#pragma unroll
          for (int k = 0; k < PER; k++) acc[k] = lane_acc[(q2 * PER + k) * 32 + lane];
          words += (lane == 0);
          bytes += (lane == 0) ? gword : 0;
          pull_finish<NW, PER>(p, app, FB, nlist, nxt, q2, w, stamp, li, lane_on && sg == 0, my_g, true, vis, acc);
        }
      }
      chunks_done = true;
    }
  }
  if (!chunks_done) {
    for (;;) {
      u64 it = 0;
      if (lane == 0) it = atomicAdd(&p.ctl->heavy_cursor[cur], 1ull);
      it = __shfl_sync(FULL_MASK, it, 0);
      // map the item number to (target state, transition group, chunk)
      u64 acc_base = 0, ci = 0;
      u32 q2s = 0, from = 0, ls = 0, js = 0;
      bool found = false;
      for (u32 q2 = 0; q2 < Q && !found; q2++)
        for (u32 j = p.q.in_begin[q2]; j < p.q.in_begin[q2 + 1]; j++) {
          const u32 l = p.q.in_label[j];
          if (!(p.q.in_from[j] & active) || l >= p.L) continue;
          const u64 cnt = p.hchunk_off[l + 1] - p.hchunk_off[l];
          if (it < acc_base + cnt) {
            found = true;
            q2s = q2;
            ls = l;
            js = j;
            from = p.q.in_from[j] & active;
            ci = p.hchunk_off[l] + (it - acc_base);
            break;
          }
          acc_base += cnt;
        }
      if (!found) break;
      const u32 *rec = p.hchunk + 3 * ci;
      const u32 w = __ldg(rec), beg = __ldg(rec + 1), end = __ldg(rec + 2);
      const u64 base = ((u64)q2s * n + w) * wpv + lane_off;
      u64 vis[PER];
      load_vis<PER>(p.vis + base, lane_on, vis);
      bool full = true;
#pragma unroll
      for (int k = 0; k < PER; k++) full &= vis[k] == ~0ull;
      if (__all_sync(FULL_MASK, full)) continue;
      u64 acc[PER];
#pragma unroll
      for (int k = 0; k < PER; k++) acc[k] = 0;
      // the sub-warps take consecutive slices of the chunk's edges
      const u32 len = end - beg, per = (len + VPW - 1) / VPW;
      const u32 sb = beg + min(len, sg * per), se = beg + min(len, (sg + 1) * per);
      u32 lfrom = from;
      if constexpr (AM == AM_GROUP) lfrom = lane_on ? p.from_tab[((u64)my_g * Q + q2s) * p.L + ls] & active : 0u;
      u32 gat = 0;
      const u32 ex = gather_row<NW, PER, EARLY, AM == AM_LANE>(p, F, bits, lfrom, sb, se, lane_off, lane_on, sg_mask,
                                                               vis, acc, gat, p.la_in_t + (u64)js * Q);
      for (u32 o = SW; o < 32; o <<= 1) {
#pragma unroll
        for (int k = 0; k < PER; k++) acc[k] |= __shfl_xor_sync(FULL_MASK, acc[k], o);
      }
      const u64 ex_all = warp_sum((u64)(li == 0 ? ex : 0));
      const u64 gat_all = warp_sum((u64)(li == 0 ? gat : 0));
      edges += (lane == 0) ? ex_all : 0;
      bytes += (lane == 0) ? 12 + gword + ex_all * (4 + (bits ? 4 * __popc(from) : 0)) + gat_all * gword : 0;
      words += (lane == 0);
      pull_finish<NW, PER>(p, app, FB, nlist, nxt, q2s, w, stamp, li, lane_on && sg == 0, my_g, true, vis, acc);
    }
  }
  append_close(p, app, nlist);
  stat[ST_PULL_EDGES] += warp_sum(edges);
  stat[ST_PULL_VERTICES] += warp_sum(words);
  stat[ST_ALG_BYTES] += warp_sum(bytes);
}

// Commit of a level: fold the new frontier words into VIS, count work, note
// the DFA states present in the new frontier, clear the old frontier words.
// set_bits: the next frontier may be sparse enough for bottom-up levels to
// test its bitmap, so its bits are set; clear_bits: this level's bits were set.
template <int NW, int AM>
__device__ void commit_phase(const BfsParams &p, int lp, u32 nxt, u64 n_cur, bool set_bits, bool clear_bits,
                             u64 *stat) {
  const u64 *list = lp ? p.list1 : p.list0;
  const u64 *nlist = lp ? p.list0 : p.list1;
  u64 *F = lp ? p.fr1 : p.fr0;
  const u64 *FB = lp ? p.fr0 : p.fr1;
  const u32 Q = p.Q;
  const u64 n_next = *(volatile unsigned long long *)&p.ctl->n_list[nxt];
  const u64 stride = (u64)gridDim.x * blockDim.x;
  const u64 tid = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  u64 W = 0, N = 0, mf = 0, gv = 0, gx = 0;
  u32 states = 0;
  for (u64 j = tid; j < n_next; j += stride) {
    u64 e = __ldcg(&nlist[j]);
    if (e == NO_ENTRY) continue;
    u32 gq = (u32)(e >> 32), w = (u32)e;
    u32 g = gq / Q, q = gq - g * Q;
    u64 wi = widx<NW>(p, g, q, w);
    Word<NW> m = load_cg<NW>(FB + wi);
    Word<NW> v = load_cg<NW>(p.vis + wi);
#pragma unroll
    for (int t = 0; t < NW; t++) v.w[t] |= m.w[t];
    store_w<NW>(p.vis + wi, v);
    if (set_bits) {
      const u64 bi = (u64)q * p.n + w;
      atomicOr(p.fbits + (lp ? 0 : p.fbits_words) + (bi >> 5), 1u << (bi & 31));
    }
    u32 c = popc_w(m);
    u32 rows = 0, d;
    if constexpr (AM == AM_LANE) {
      d = la_degsum<NW>(p, q, w, g, m, W, &rows);
    } else {
      d = degsum(p, gdesc<AM>(p, g), q, w, &rows);
      W += (u64)c * d;
    }
    N += c;
    mf += d;
    gx += rows;
    gv += 1;
    states |= 1u << q;
  }
  Word<NW> zero;
#pragma unroll
  for (int t = 0; t < NW; t++) zero.w[t] = 0;
  for (u64 j = tid; j < n_cur; j += stride) {
    u64 e = __ldcg(&list[j]);
    if (e == NO_ENTRY) continue;
    u32 gq = (u32)(e >> 32);
    u32 g = gq / Q;
    store_w<NW>(F + widx<NW>(p, g, gq - g * Q, (u32)e), zero);
    if (clear_bits) {
      // the retired frontier's bitmap: every set bit belongs to one of these entries
      const u64 bi = (u64)(gq - g * Q) * p.n + (u32)e;
      p.fbits[(lp ? p.fbits_words : 0) + (bi >> 5)] = 0u;
    }
  }
  if (tid == 0) stat[ST_ALG_BYTES] += n_cur * (8 + 8 * NW);
  W = warp_sum(W);
  N = warp_sum(N);
  mf = warp_sum(mf);
  gv = warp_sum(gv);
  gx = warp_sum(gx);
  states = __reduce_or_sync(FULL_MASK, states);
  // per new entry: the entry, its new frontier word, its visited word read and
  // written; per old entry: the entry and its frontier word cleared
  if (lane_id() == 0) stat[ST_ALG_BYTES] += gv * (8 + 24 * NW);
  if (lane_id() == 0) {
    stat[ST_W] += W;
    stat[ST_N] += N;
    stat[ST_GROUP_VERTICES] += gv;
    if (mf) atomicAdd(&p.ctl->stats[ST_GROUP_W], mf);
    if (gx) atomicAdd(&p.ctl->stats[ST_GROUP_X], gx);
    if (mf) atomicAdd(&p.ctl->mf[nxt], mf);
    if (states) atomicOr(&p.ctl->smask[nxt], states);
  }
}

// Bytes a bottom-up level moves when the frontier holds the states `active`:
// per target state with an active incoming transition, its visited words;
// per such transition group, the row offsets and per in-edge a column id
// and the gathered frontier words.
template <int NW>
__device__ double pull_bytes(const BfsParams &p, u32 active) {
  double b = 0;
  const double wv = 8.0 * NW * p.G;
  for (u32 q2 = 0; q2 < p.Q; q2++) {
    bool any = false;
    for (u32 j = p.q.in_begin[q2]; j < p.q.in_begin[q2 + 1]; j++) {
      const u32 f = p.q.in_from[j] & active, l = p.q.in_label[j];
      if (!f || l >= p.L) continue;
      any = true;
      b += 8.0 * p.n + (double)p.label_edges[l] * (4.0 + wv * __popc(f));
    }
    if (any) b += wv * p.n;
  }
  return b;
}

template <int NW, int AM>
__global__ void __launch_bounds__(BFS_THREADS, 4) msbfs_kernel(const __grid_constant__ BfsParams p) {
  // per-warp statistics, summed into the control block at the end
  u64 stat[ST_COUNT];
#pragma unroll
  for (int i = 0; i < ST_COUNT; i++) stat[i] = 0;
  BfsCtl *c = p.ctl;
  const bool tracer = blockIdx.x == 0 && threadIdx.x == 0;

  seed_phase<NW, AM>(p, stat);
  if (!grid_barrier(c, p.nblocks, p.time_limit_ns)) return;

  u32 level = 0;
  for (;; level++) {
    const u32 cur = level % 3, nxt = (level + 1) % 3, old = (level + 2) % 3;
    const int lp = level & 1;
    const u64 n_cur = *(volatile unsigned long long *)&c->n_list[cur];
    if (n_cur == 0) break;
    const u64 mf = *(volatile unsigned long long *)&c->mf[cur];
    const u32 active = *(volatile unsigned *)&c->smask[cur];
    const double push_cost = (double)mf * (4.0 + 8.0 * NW) + (double)n_cur * (16.0 + 8.0 * NW);
    const bool push = p.force == 1 || (p.force != 2 && (double)p.alpha * push_cost < pull_bytes<NW>(p, active));
    if (tracer) {
      // counters of the level after next start at zero
      c->n_list[old] = 0;
      c->cursor[old] = 0;
      c->mf[old] = 0;
      c->spill_count[old] = 0;
      c->spill_cursor[old] = 0;
      c->heavy_cursor[old] = 0;
      c->smask[old] = 0;
      if (level < (u32)TRACE_LEVELS) {
        c->trace_t[level] = globaltimer_ns();
        c->trace_n[level] = n_cur;
        c->trace_mode[level] = push ? 1u : 2u;
        c->trace_mf[level] = mf;
      }
      if (push)
        stat[ST_PUSH_LEVELS] += 1;
      else
        stat[ST_PULL_LEVELS] += 1;
    }
    const u32 stamp = p.stamp_base + level + 2;  // the seeds used stamp_base + 1
    if (push) {
      push_level<NW, AM>(p, lp, cur, nxt, n_cur, stamp, stat);
      if (!grid_barrier(c, p.nblocks, p.time_limit_ns)) return;
      if (*(volatile unsigned long long *)&c->spill_count[cur] != 0) {
        spill_phase<NW>(p, lp, cur, nxt, stamp, stat);
        if (!grid_barrier(c, p.nblocks, p.time_limit_ns)) return;
      }
    } else {
      // a sparse frontier: test the frontier bitmap before each gather
      // (implies n_cur * 4 < n * Q, so the commit that built this frontier set its bits)
      const bool sparse = p.fbits && n_cur * 4 < (u64)p.n * __popc(active);
      const u32 *bits = sparse ? p.fbits + (lp ? p.fbits_words : 0) : nullptr;
      // early exit pays where few lanes are live: one lane group, the
      // per-group automata of a multi launch (typically one start vertex
      // each), or per-lane automata (lanes of short queries go quiet early)
      if (p.G == 1 || AM != AM_ONE)
        pull_level<NW, true, AM>(p, lp, cur, nxt, active, stamp, bits, stat);
      else
        pull_level<NW, false, AM>(p, lp, cur, nxt, active, stamp, bits, stat);
      if (!grid_barrier(c, p.nblocks, p.time_limit_ns)) return;
    }
    {
      // bitmaps only where a bottom-up level may test them: a frontier with
      // fewer than n * Q / 4 entries (the seeds always set theirs)
      const u64 n_next = *(volatile unsigned long long *)&c->n_list[nxt];
      const u64 sparse_cap = (u64)p.n * p.Q;
      const bool set_bits = p.fbits && n_next * 4 < sparse_cap;
      const bool clear_bits = p.fbits && (level == 0 || n_cur * 4 < sparse_cap);
      if (tracer && level < (u32)TRACE_LEVELS) c->trace_c[level] = globaltimer_ns();
      commit_phase<NW, AM>(p, lp, nxt, n_cur, set_bits, clear_bits, stat);
    }
    if (!grid_barrier(c, p.nblocks, p.time_limit_ns)) return;
  }
  if (lane_id() == 0) {
#pragma unroll
    for (int i = 0; i < ST_COUNT; i++)
      if (stat[i]) atomicAdd(&c->stats[i], stat[i]);
  }
  if (tracer) {
    c->levels = level;
    c->trace_t[level < (u32)TRACE_LEVELS ? level : TRACE_LEVELS] = globaltimer_ns();
  }
}

// VIS words start as the mask of empty lanes of their group, so empty lanes
// look visited everywhere (this also lets bottom-up levels stop early).
template <int NW>
__global__ void vis_init_kernel(u64 *__restrict__ vis, u64 total, u32 G, const u64 *__restrict__ empty) {
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (u64)gridDim.x * blockDim.x) {
    u32 g = (u32)((i / NW) % G);
    vis[i] = empty[(u64)g * NW + (i % NW)];
  }
}

cudaError_t launch_vis_init(int nw, const BfsParams &p, const unsigned long long *empty, cudaStream_t st) {
  u64 total = (u64)p.Q * p.n * p.G * nw;
  u64 blocks = (total + 255) / 256;
  if (blocks > 152ull * 32) blocks = 152ull * 32;
  if (blocks == 0) blocks = 1;
  if (nw == 1)
    vis_init_kernel<1><<<(unsigned)blocks, 256, 0, st>>>(p.vis, total, p.G, empty);
  else
    vis_init_kernel<4><<<(unsigned)blocks, 256, 0, st>>>(p.vis, total, p.G, empty);
  return cudaGetLastError();
}

// Lane mode: VIS words start as empty_q[(q * G + g) * NW + k], the lanes that
// are empty or whose automaton has no state q (so they look visited there).
template <int NW>
__global__ void vis_init_lane_kernel(u64 *__restrict__ vis, u64 total, u64 per_state, u32 G,
                                     const u64 *__restrict__ empty_q) {
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (u64)gridDim.x * blockDim.x) {
    const u64 q = i / per_state;
    const u32 gk = (u32)(i % ((u64)G * NW));
    vis[i] = empty_q[q * G * NW + gk];
  }
}

cudaError_t launch_vis_init_lane(int nw, const BfsParams &p, const unsigned long long *empty_q, cudaStream_t st) {
  const u64 per_state = (u64)p.n * p.G * nw;
  const u64 total = per_state * p.Q;
  u64 blocks = (total + 255) / 256;
  if (blocks > 152ull * 32) blocks = 152ull * 32;
  if (blocks == 0) blocks = 1;
  if (nw == 1)
    vis_init_lane_kernel<1><<<(unsigned)blocks, 256, 0, st>>>(p.vis, total, per_state, p.G, empty_q);
  else
    vis_init_lane_kernel<4><<<(unsigned)blocks, 256, 0, st>>>(p.vis, total, per_state, p.G, empty_q);
  return cudaGetLastError();
}

// flag[i] = 1 when start vertex srcs[i] has an edge on a label of label_mask
// in the traversal's forward direction (off = the forward offsets).
__global__ void source_filter_kernel(const u32 *__restrict__ off, u32 n, u32 L, unsigned long long label_mask,
                                     const u32 *__restrict__ srcs, u64 count, unsigned char *__restrict__ flag) {
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (u64)gridDim.x * blockDim.x) {
    const u32 s = srcs[i];
    unsigned char f = 0;
    for (unsigned long long m = label_mask; m && !f; m &= m - 1) {
      const u32 l = __ffsll(m) - 1;
      if (l >= L) break;
      const u32 *o = off + (u64)l * (n + 1) + s;
      f = __ldg(o + 1) > __ldg(o);
    }
    flag[i] = f;
  }
}

cudaError_t launch_source_filter(const uint32_t *off, uint32_t n, uint32_t L, unsigned long long label_mask,
                                 const uint32_t *srcs, unsigned long long count, unsigned char *flag,
                                 cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  u64 blocks = (count + 255) / 256;
  if (blocks > 152ull * 16) blocks = 152ull * 16;
  source_filter_kernel<<<(unsigned)blocks, 256, 0, st>>>(off, n, L, label_mask, srcs, count, flag);
  return cudaGetLastError();
}

cudaError_t launch_msbfs(int nw, const BfsParams &p, int blocks, int threads, cudaStream_t st) {
  void *args[] = {(void *)&p};
  if (nw == 1)
    return cudaLaunchCooperativeKernel((void *)msbfs_kernel<1, AM_ONE>, blocks, threads, args, 0, st);
  return cudaLaunchCooperativeKernel((void *)msbfs_kernel<4, AM_ONE>, blocks, threads, args, 0, st);
}

int msbfs_max_blocks(int nw, int threads, int *blocks_per_sm, int *sms) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e;
  if (nw == 1)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, msbfs_kernel<1, AM_ONE>, threads, 0);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, msbfs_kernel<4, AM_ONE>, threads, 0);
  return e == cudaSuccess ? 0 : -1;
}

cudaError_t preload_static_msbfs_kernels() {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, msbfs_kernel<1, AM_ONE>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, vis_init_kernel<1>);
  return e;
}

cudaError_t launch_msbfs_multi(const BfsParams &p, int blocks, int threads, cudaStream_t st) {
  void *args[] = {(void *)&p};
  return cudaLaunchCooperativeKernel((void *)msbfs_kernel<1, AM_GROUP>, blocks, threads, args, 0, st);
}

cudaError_t launch_msbfs_lane(int nw, const BfsParams &p, int blocks, int threads, cudaStream_t st) {
  void *args[] = {(void *)&p};
  if (nw == 1)
    return cudaLaunchCooperativeKernel((void *)msbfs_kernel<1, AM_LANE>, blocks, threads, args, 0, st);
  return cudaLaunchCooperativeKernel((void *)msbfs_kernel<4, AM_LANE>, blocks, threads, args, 0, st);
}

int msbfs_lane_max_blocks(int nw, int threads, int *blocks_per_sm) {
  cudaError_t e;
  if (nw == 1)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, msbfs_kernel<1, AM_LANE>, threads, 0);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, msbfs_kernel<4, AM_LANE>, threads, 0);
  return e == cudaSuccess ? 0 : -1;
}

int msbfs_multi_max_blocks(int threads, int *blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, msbfs_kernel<1, AM_GROUP>, threads, 0) ==
                 cudaSuccess
             ? 0
             : -1;
}

}  // namespace rpq
