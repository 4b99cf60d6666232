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
// lane group.  For every (group, state, vertex) there is one K-bit word in
// each of three arrays: VIS (visited), and two frontier words used in
// ping-pong.  One word operation therefore advances K searches.  A level is
// expanded either
//   * top-down ("push"): the sparse list of frontier entries is scanned, each
//     entry's out-edges on the labels of its state's transitions are read and
//     the new lanes are OR-ed into the next frontier word with atomics, or
//   * bottom-up ("pull"): every (vertex, target state) word gathers the
//     frontier words of its in-neighbours on the transition labels, with no
//     atomics and an early exit once all lanes are visited,
// chosen per level from the byte cost of each.  The whole search is one
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
__device__ __forceinline__ bool all_bits(const Word<NW> &x) {
  u64 a = ~0ull;
#pragma unroll
  for (int i = 0; i < NW; i++) a &= x.w[i];
  return a == ~0ull;
}

template <int NW>
__device__ __forceinline__ u32 popc_w(const Word<NW> &x) {
  u32 c = 0;
#pragma unroll
  for (int i = 0; i < NW; i++) c += __popcll(x.w[i]);
  return c;
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

// Out-degree of v summed over the labels leaving DFA state q.
__device__ __forceinline__ u32 degsum(const BfsParams &p, u32 q, u32 v) {
  u32 s = 0;
  const u32 n1 = p.n + 1;
  for (u32 t = p.q.out_begin[q]; t < p.q.out_begin[q + 1]; t++) {
    u32 l = p.q.out_label[t];
    if (l >= p.L) continue;
    const u32 *off = p.out_off + (u64)l * n1 + v;
    s += __ldg(off + 1) - __ldg(off);
  }
  return s;
}

// Warp-aggregated append of `entry` for the lanes with `take` set.  All 32
// lanes must call it.
__device__ __forceinline__ void warp_append(bool take, u64 entry, unsigned long long *count, u64 *list) {
  u32 b = __ballot_sync(FULL_MASK, take);
  if (!b) return;
  u64 base = 0;
  if (lane_id() == __ffs(b) - 1) base = atomicAdd(count, (unsigned long long)__popc(b));
  base = __shfl_sync(FULL_MASK, base, __ffs(b) - 1);
  if (take) list[base + __popc(b & lanemask_lt())] = entry;
}

template <int NW>
__device__ void seed_phase(const BfsParams &p, u64 *stat) {
  const u32 K = 64 * NW;
  const u64 total = (u64)p.G * K;
  const u64 stride = (u64)gridDim.x * blockDim.x;
  u64 W = 0, N = 0, mf = 0;
  for (u64 base = (u64)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < total; base += stride) {
    u64 i = base + lane_id();
    bool take = false;
    u64 entry = 0;
    if (i < total) {
      u32 s = p.lanesrc[i];
      if (s != NO_SOURCE) {
        u32 g = (u32)(i / K), lane = (u32)(i % K);
        u64 gq = (u64)g * p.Q;  // start state 0
        u64 wi = (gq * p.n + s) * NW;
        p.vis[wi + lane / 64] |= 1ull << (lane % 64);
        p.fr0[wi + lane / 64] = 1ull << (lane % 64);
        entry = (gq << 32) | s;
        take = true;
        u32 d = degsum(p, 0, s);
        W += d;
        N += 1;
        mf += d;
      }
    }
    warp_append(take, entry, &p.ctl->n_list[0], p.list0);
  }
  W = warp_sum(W);
  N = warp_sum(N);
  mf = warp_sum(mf);
  if (lane_id() == 0) {
    stat[ST_W] += W;
    stat[ST_N] += N;
    stat[ST_GROUP_VERTICES] += N;
    if (mf) atomicAdd(&p.ctl->mf[0], mf);
  }
}

// Top-down expansion of the entries of the current list.
template <int NW>
__device__ void push_level(const BfsParams &p, int lp, u32 cur, u32 nxt, u64 n_cur, u32 stamp, u64 *stat) {
  const u64 *list = lp ? p.list1 : p.list0;
  u64 *nlist = lp ? p.list0 : p.list1;
  const u64 *F = lp ? p.fr1 : p.fr0;
  u64 *FB = lp ? p.fr0 : p.fr1;
  const u32 n = p.n, Q = p.Q, n1 = p.n + 1;
  const u32 lane = lane_id();
  u64 edges = 0, rows = 0;
  for (;;) {
    u64 base = 0;
    if (lane == 0) base = atomicAdd(&p.ctl->cursor[cur], 32ull);
    base = __shfl_sync(FULL_MASK, base, 0);
    if (base >= n_cur) break;
    u64 idx = base + lane;
    bool valid = idx < n_cur;
    u64 e = valid ? __ldcg(&list[idx]) : 0;
    u32 gq = (u32)(e >> 32), v = (u32)e;
    u32 g = gq / Q, q = gq - g * Q;
    Word<NW> fm;
#pragma unroll
    for (int i = 0; i < NW; i++) fm.w[i] = 0;
    if (valid) fm = load_cg<NW>(F + ((u64)gq * n + v) * NW);
    u32 t_beg = valid ? p.q.out_begin[q] : 0;
    u32 nt = valid ? p.q.out_begin[q + 1] - t_beg : 0;
    u32 max_nt = __reduce_max_sync(FULL_MASK, nt);
    for (u32 j = 0; j < max_nt; j++) {
      u32 rbeg = 0, rlen = 0, tgq = 0;
      if (j < nt) {
        u32 t = t_beg + j;
        u32 l = p.q.out_label[t];
        tgq = g * Q + p.q.out_to[t];
        if (l < p.L) {
          const u32 *off = p.out_off + (u64)l * n1 + v;
          rbeg = __ldg(off);
          rlen = __ldg(off + 1) - rbeg;
          rows++;
        }
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
        for (int i = 0; i < NW; i++) ofm.w[i] = __shfl_sync(FULL_MASK, fm.w[i], o);
        bool take = false;
        u32 w = 0;
        if (k < total) {
          w = __ldg(p.out_col + o_beg + (k - o_pre));
          u64 wi = ((u64)o_gq * n + w) * NW;
          Word<NW> vis = load_cg<NW>(p.vis + wi);
          Word<NW> m;
#pragma unroll
          for (int i = 0; i < NW; i++) m.w[i] = ofm.w[i] & ~vis.w[i];
          if (any_bits(m)) {
            if constexpr (NW == 1) {
              u64 old = atomicOr((unsigned long long *)(FB + wi), m.w[0]);
              take = (old == 0);
            } else {
#pragma unroll
              for (int i = 0; i < NW; i++)
                if (m.w[i]) atomicOr((unsigned long long *)(FB + wi + i), m.w[i]);
              u32 old = atomicMax(p.claim + ((u64)o_gq * n + w), stamp);
              take = old < stamp;
            }
          }
        }
        warp_append(take, ((u64)o_gq << 32) | w, &p.ctl->n_list[nxt], nlist);
      }
    }
  }
  stat[ST_GROUP_EDGES] += warp_sum(edges);
  stat[ST_GROUP_ROWS] += warp_sum(rows);
}

// Bottom-up expansion over every (group, vertex).
template <int NW>
__device__ void pull_level(const BfsParams &p, int lp, u32 nxt, u64 *stat) {
  const u64 *F = lp ? p.fr1 : p.fr0;
  u64 *FB = lp ? p.fr0 : p.fr1;
  u64 *nlist = lp ? p.list0 : p.list1;
  const u32 n = p.n, Q = p.Q, n1 = p.n + 1;
  const u64 total = (u64)p.G * n;
  const u64 stride = (u64)gridDim.x * blockDim.x;
  u64 edges = 0, words = 0;
  for (u64 base = (u64)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < total; base += stride) {
    u64 item = base + lane_id();
    bool valid = item < total;
    u32 g = valid ? (u32)(item / n) : 0;
    u32 w = valid ? (u32)(item - (u64)g * n) : 0;
    // high in-degree vertices are left to the warp-per-vertex loop below
    if (valid && p.heavy_bits && (__ldg(p.heavy_bits + (w >> 5)) >> (w & 31) & 1u)) valid = false;
    for (u32 q2 = 0; q2 < Q; q2++) {
      u32 gb = p.q.in_begin[q2], ge = p.q.in_begin[q2 + 1];
      if (gb == ge) continue;
      bool take = false;
      u64 gq2 = (u64)g * Q + q2;
      bool has_in = false;  // skip vertices with no in-edge on these labels
      if (valid)
        for (u32 j = gb; j < ge && !has_in; j++) {
          u32 l = p.q.in_label[j];
          if (l >= p.L) continue;
          const u32 *off = p.in_off + (u64)l * n1 + w;
          has_in = __ldg(off) != __ldg(off + 1);
        }
      if (has_in) {
        u64 wi = (gq2 * n + w) * NW;
        Word<NW> vis = load_cg<NW>(p.vis + wi);
        if (!all_bits(vis)) {
          words++;
          Word<NW> acc;
#pragma unroll
          for (int i = 0; i < NW; i++) acc.w[i] = 0;
          bool full = false;
          for (u32 j = gb; j < ge && !full; j++) {
            u32 l = p.q.in_label[j];
            if (l >= p.L) continue;
            u32 from = p.q.in_from[j];
            const u32 *off = p.in_off + (u64)l * n1 + w;
            u32 beg = __ldg(off), end = __ldg(off + 1);
            for (u32 i = beg; i < end; i++) {
              u32 v = __ldg(p.in_col + i);
              edges++;
              for (u32 fb = from; fb; fb &= fb - 1) {
                u32 q = __ffs(fb) - 1;
                Word<NW> f = load_cg<NW>(F + (((u64)g * Q + q) * n + v) * NW);
#pragma unroll
                for (int t = 0; t < NW; t++) acc.w[t] |= f.w[t];
              }
              Word<NW> cover;
#pragma unroll
              for (int t = 0; t < NW; t++) cover.w[t] = acc.w[t] | vis.w[t];
              if (all_bits(cover)) {
                full = true;
                break;
              }
            }
          }
          Word<NW> nw;
#pragma unroll
          for (int t = 0; t < NW; t++) nw.w[t] = acc.w[t] & ~vis.w[t];
          if (any_bits(nw)) {
            Word<NW> nv;
#pragma unroll
            for (int t = 0; t < NW; t++) nv.w[t] = vis.w[t] | nw.w[t];
            store_w<NW>(p.vis + wi, nv);
            store_w<NW>(FB + wi, nw);
            take = true;
          }
        }
      }
      warp_append(take, (gq2 << 32) | w, &p.ctl->n_list[nxt], nlist);
    }
  }
  // High in-degree vertices: a warp per (group, vertex); lanes stride over
  // the in-edges and the partial words are OR-reduced across the warp.
  const u64 n_hv = (u64)p.G * p.n_heavy;
  const u32 lane = lane_id();
  for (u64 it = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < n_hv; it += stride >> 5) {
    const u32 g = (u32)(it / p.n_heavy);
    const u32 w = __ldg(p.heavy_list + (it - (u64)g * p.n_heavy));
    for (u32 q2 = 0; q2 < Q; q2++) {
      u32 gb = p.q.in_begin[q2], ge = p.q.in_begin[q2 + 1];
      if (gb == ge) continue;
      const u64 gq2 = (u64)g * Q + q2;
      const u64 wi = (gq2 * n + w) * NW;
      Word<NW> vis = load_cg<NW>(p.vis + wi);
      if (all_bits(vis)) continue;
      Word<NW> acc;
#pragma unroll
      for (int t = 0; t < NW; t++) acc.w[t] = 0;
      for (u32 j = gb; j < ge; j++) {
        u32 l = p.q.in_label[j];
        if (l >= p.L) continue;
        u32 from = p.q.in_from[j];
        const u32 *off = p.in_off + (u64)l * n1 + w;
        u32 beg = __ldg(off), end = __ldg(off + 1);
        for (u32 i = beg + lane; i < end; i += 32) {
          u32 v = __ldg(p.in_col + i);
          edges++;
          for (u32 fb = from; fb; fb &= fb - 1) {
            u32 q = __ffs(fb) - 1;
            Word<NW> f = load_cg<NW>(F + (((u64)g * Q + q) * n + v) * NW);
#pragma unroll
            for (int t = 0; t < NW; t++) acc.w[t] |= f.w[t];
          }
        }
      }
#pragma unroll
      for (int t = 0; t < NW; t++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc.w[t] |= __shfl_xor_sync(FULL_MASK, acc.w[t], o);
      Word<NW> nw;
#pragma unroll
      for (int t = 0; t < NW; t++) nw.w[t] = acc.w[t] & ~vis.w[t];
      bool take = false;
      if (lane == 0) {
        words++;
        if (any_bits(nw)) {
          Word<NW> nv;
#pragma unroll
          for (int t = 0; t < NW; t++) nv.w[t] = vis.w[t] | nw.w[t];
          store_w<NW>(p.vis + wi, nv);
          store_w<NW>(FB + wi, nw);
          take = true;
        }
      }
      warp_append(take, (gq2 << 32) | w, &p.ctl->n_list[nxt], nlist);
    }
  }
  stat[ST_PULL_EDGES] += warp_sum(edges);
  stat[ST_PULL_VERTICES] += warp_sum(words);
}

// Commit of a level: fold the new frontier into VIS (top-down levels), count
// work, clear the old frontier words.
template <int NW>
__device__ void commit_phase(const BfsParams &p, int lp, u32 nxt, u64 n_cur, bool was_push, u64 *stat) {
  const u64 *list = lp ? p.list1 : p.list0;
  const u64 *nlist = lp ? p.list0 : p.list1;
  u64 *F = lp ? p.fr1 : p.fr0;
  const u64 *FB = lp ? p.fr0 : p.fr1;
  const u32 n = p.n, Q = p.Q;
  const u64 n_next = *(volatile unsigned long long *)&p.ctl->n_list[nxt];
  const u64 stride = (u64)gridDim.x * blockDim.x;
  const u64 tid = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  u64 W = 0, N = 0, mf = 0, gv = 0;
  for (u64 j = tid; j < n_next; j += stride) {
    u64 e = __ldcg(&nlist[j]);
    u32 gq = (u32)(e >> 32), w = (u32)e;
    u32 q = gq % Q;
    u64 wi = ((u64)gq * n + w) * NW;
    Word<NW> m = load_cg<NW>(FB + wi);
    if (was_push) {
      Word<NW> v = load_cg<NW>(p.vis + wi);
#pragma unroll
      for (int t = 0; t < NW; t++) v.w[t] |= m.w[t];
      store_w<NW>(p.vis + wi, v);
    }
    u32 c = popc_w(m);
    u32 d = degsum(p, q, w);
    W += (u64)c * d;
    N += c;
    mf += d;
    gv += 1;
  }
  Word<NW> zero;
#pragma unroll
  for (int t = 0; t < NW; t++) zero.w[t] = 0;
  for (u64 j = tid; j < n_cur; j += stride) {
    u64 e = __ldcg(&list[j]);
    u64 wi = ((u64)(u32)(e >> 32) * n + (u32)e) * NW;
    store_w<NW>(F + wi, zero);
  }
  W = warp_sum(W);
  N = warp_sum(N);
  mf = warp_sum(mf);
  gv = warp_sum(gv);
  if (lane_id() == 0) {
    stat[ST_W] += W;
    stat[ST_N] += N;
    stat[ST_GROUP_VERTICES] += gv;
    if (mf) atomicAdd(&p.ctl->mf[nxt], mf);
  }
}

template <int NW>
__global__ void __launch_bounds__(BFS_THREADS) msbfs_kernel(const __grid_constant__ BfsParams p) {
  // per-warp statistics, summed into the control block at the end
  u64 stat[ST_COUNT];
#pragma unroll
  for (int i = 0; i < ST_COUNT; i++) stat[i] = 0;
  BfsCtl *c = p.ctl;

  seed_phase<NW>(p, stat);
  if (!grid_barrier(c, p.nblocks, p.time_limit_ns)) return;

  u32 level = 0;
  for (;; level++) {
    const u32 cur = level % 3, nxt = (level + 1) % 3, old = (level + 2) % 3;
    const int lp = level & 1;
    const u64 n_cur = *(volatile unsigned long long *)&c->n_list[cur];
    if (n_cur == 0) break;
    const u64 mf = *(volatile unsigned long long *)&c->mf[cur];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      c->n_list[old] = 0;
      c->cursor[old] = 0;
      c->mf[old] = 0;
    }
    const double push_cost = (double)mf * (4.0 + 8.0 * NW) + (double)n_cur * (16.0 + 8.0 * NW);
    const bool push = p.force == 1 || (p.force != 2 && (double)p.alpha * push_cost < p.pull_cost_fixed);
    if (push) {
      push_level<NW>(p, lp, cur, nxt, n_cur, p.stamp_base + level + 1, stat);
    } else {
      pull_level<NW>(p, lp, nxt, stat);
    }
    if (threadIdx.x == 0 && blockIdx.x == 0) stat[push ? ST_PUSH_LEVELS : ST_PULL_LEVELS] += 1;
    if (!grid_barrier(c, p.nblocks, p.time_limit_ns)) return;
    commit_phase<NW>(p, lp, nxt, n_cur, push, stat);
    if (!grid_barrier(c, p.nblocks, p.time_limit_ns)) return;
  }
  if (lane_id() == 0) {
#pragma unroll
    for (int i = 0; i < ST_COUNT; i++)
      if (stat[i]) atomicAdd(&c->stats[i], stat[i]);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) c->levels = level;
}

// VIS words start as the mask of empty lanes of their group, so empty lanes
// look visited everywhere (this also lets bottom-up levels stop early).
template <int NW>
__global__ void vis_init_kernel(u64 *__restrict__ vis, u64 words_per_group, u32 G,
                                const u64 *__restrict__ empty) {
  u64 total = words_per_group * G;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (u64)gridDim.x * blockDim.x) {
    u32 g = (u32)(i / words_per_group);
    vis[i] = empty[(u64)g * NW + (i % NW)];
  }
}

cudaError_t launch_vis_init(int nw, const BfsParams &p, const unsigned long long *empty, cudaStream_t st) {
  u64 wpg = (u64)p.Q * p.n * nw;
  u64 total = wpg * p.G;
  u64 blocks = (total + 255) / 256;
  if (blocks > 152ull * 32) blocks = 152ull * 32;
  if (blocks == 0) blocks = 1;
  if (nw == 1)
    vis_init_kernel<1><<<(unsigned)blocks, 256, 0, st>>>(p.vis, wpg, p.G, empty);
  else
    vis_init_kernel<4><<<(unsigned)blocks, 256, 0, st>>>(p.vis, wpg, p.G, empty);
  return cudaGetLastError();
}

cudaError_t launch_msbfs(int nw, const BfsParams &p, int blocks, int threads, cudaStream_t st) {
  void *args[] = {(void *)&p};
  if (nw == 1)
    return cudaLaunchCooperativeKernel((void *)msbfs_kernel<1>, blocks, threads, args, 0, st);
  return cudaLaunchCooperativeKernel((void *)msbfs_kernel<4>, blocks, threads, args, 0, st);
}

int msbfs_max_blocks(int nw, int threads, int *blocks_per_sm, int *sms) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e;
  if (nw == 1)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, msbfs_kernel<1>, threads, 0);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, msbfs_kernel<4>, threads, 0);
  return e == cudaSuccess ? 0 : -1;
}

}  // namespace rpq
