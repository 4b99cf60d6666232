// CRPQ evaluation (Definition 2, Section 2.1) on the device.
//
// The paper materializes the result of every RPQ atom and combines them with
// a worst-case optimal join, choosing per atom the direction the matching
// order needs (Section 6.3).  This module does the same kind of join,
// variable at a time, with all data on the device:
//
//   * Variables are bound in a fixed order that starts with variable 0 (whose
//     values are processed in batches, so batches come out in order) and then
//     repeatedly takes the variable with the most atoms to bound variables.
//   * Each atom constrains the later-bound of its two variables.  An atom
//     x -rho-> y whose x is bound first is evaluated forward from the distinct
//     bound x values; one whose y is bound first is evaluated from the target
//     end (reversed language over in-edges) from the distinct y values.  Both
//     give, per bound value, a sorted row of admissible values for the new
//     variable.  A self-loop atom x -rho-> x is checked once x is bound.
//     Rows are referenced where the emission wrote them; a row holding at
//     least crpq_bitset_frac of the vertices is also written as a bitset over
//     the vertices (a direct-address membership table).
//   * Binding a variable: per partial tuple, the constraint with the shortest
//     listed row generates the candidates (the smallest-first intersection of
//     worst case optimal joins); every other constraint is a membership test,
//     one load in a bitset or a binary search in a sorted row; vertex labels
//     are tested too.  The surviving (tuple, value) pairs are compacted into
//     the next table.  Candidates are processed in slices of bounded size.
//   * The last variable of a count-only query (no self-loop on it) is bound,
//     counted and digested in one pass (count_last_kernel); its long rows are
//     kept as bitsets only, and a tuple whose rows are all bitsets is
//     extended by a word-by-word AND of them.
//   * Complete tuples of a batch are sorted lexicographically in declaration
//     order (stable LSD passes over the columns) and digested.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <numeric>
#include <vector>

#include "crpq.h"

namespace rpq {
namespace {

constexpr uint64_t CAND_CAP = 1ull << 26;  // candidate pairs per expansion slice
constexpr uint32_t BATCH0 = 4096;          // values of variable 0 per batch
constexpr int MAXC = RPQ_MAX_ATOMS;

struct DevRows {  // rows of one atom for a sorted set of endpoint values
  const u32 *src;   // the values with a row, ascending
  const u64 *ptr;   // per row: device address of its sorted destinations
  const u64 *bptr;  // per row: device address of its bitset over the vertices, or 0
  const u32 *len;   // per row: its number of destinations
  u32 ns;
};

struct Cons {
  DevRows rows;
  const u32 *col;  // bound endpoint's column; nullptr: the variable being bound
};

struct StepParams {
  u32 nc;
  u32 gen_mask;  // constraints that may generate candidates
  int want_label;
  const uint8_t *vlabel;
  // count-only last step: rows with a bitset have no list (they generate no
  // candidates), and a tuple whose rows all have bitsets is joined word by
  // word (DENSE); lbits = the vertices of label want_label as a bitset
  u32 fused;
  u64 bwords;
  const u64 *lbits;
  Cons c[MAXC];
};

constexpr uint8_t DENSE = 0x80;  // flag in a tuple's generator byte

struct ColPtrs {
  const u32 *in[RPQ_MAX_VARS];
  u32 *out[RPQ_MAX_VARS + 1];
};

// Row of value v: its destinations (sorted; nullptr when the row is kept as
// a bitset only) and their number (0 if v has no row); returns the row's
// bitset, or nullptr when it has none.
__device__ __forceinline__ const u64 *lookup(const DevRows &r, u32 v, const u32 **row, u32 *l) {
  u32 lo = 0, hi = r.ns;
  while (lo < hi) {
    u32 mid = (lo + hi) >> 1;
    u32 s = r.src[mid];
    if (s < v)
      lo = mid + 1;
    else
      hi = mid;
  }
  if (lo < r.ns && r.src[lo] == v) {
    *row = reinterpret_cast<const u32 *>(r.ptr[lo]);
    *l = r.len[lo];
    return reinterpret_cast<const u64 *>(r.bptr[lo]);
  }
  *row = nullptr;
  *l = 0;
  return nullptr;
}

__device__ __forceinline__ bool row_has(const u32 *row, u32 l, u32 y) {
  u32 lo = 0, hi = l;
  while (lo < hi) {
    u32 mid = (lo + hi) >> 1;
    u32 s = row[mid];
    if (s < y)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo < l && row[lo] == y;
}

// y in the row (its bitset when it has one, else its sorted destinations)?
__device__ __forceinline__ bool member(const u32 *row, u32 l, const u64 *bits, u32 y) {
  if (bits) return (bits[y >> 6] >> (y & 63)) & 1ull;
  return row_has(row, l, y);
}

// Per tuple: the generating constraint (shortest listed row) and its length;
// in a fused step, DENSE when every row of the tuple is a bitset.
__global__ void choose_gen(const StepParams p, u64 nT, u32 *__restrict__ cnt, uint8_t *__restrict__ which) {
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < nT; i += (u64)gridDim.x * blockDim.x) {
    u32 best = 0xffffffffu, w = 0xff;
    bool all_bits = p.fused != 0;
    for (u32 k = 0; k < p.nc; k++) {
      if (!(p.gen_mask >> k & 1u)) continue;
      const u32 *row;
      u32 l;
      const u64 *bits = lookup(p.c[k].rows, p.c[k].col[i], &row, &l);
      if (p.fused && bits) continue;  // bitset only
      all_bits = false;
      if (l < best) {
        best = l;
        w = k;
      }
    }
    if (all_bits) {
      cnt[i] = 0;
      which[i] = DENSE;
    } else {
      cnt[i] = (w == 0xff) ? 0u : best;
      which[i] = (uint8_t)w;
    }
  }
}

// Candidates first .. first+n-1 of the expansion (global candidate index j
// belongs to the tuple i with off[i] <= j < off[i+1]).
__global__ void expand_cands(const StepParams p, u64 nT, const u64 *__restrict__ off,
                             const uint8_t *__restrict__ which, u64 first, u64 n, u32 *__restrict__ cand_t,
                             u32 *__restrict__ cand_v) {
  for (u64 k = (u64)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (u64)gridDim.x * blockDim.x) {
    u64 j = first + k;
    u64 lo = 0, hi = nT;  // off[lo] <= j < off[hi]
    while (hi - lo > 1) {
      u64 mid = (lo + hi) >> 1;
      if (off[mid] <= j)
        lo = mid;
      else
        hi = mid;
    }
    const Cons &c = p.c[which[lo]];
    const u32 *row;
    u32 l;
    lookup(c.rows, c.col[lo], &row, &l);
    cand_t[k] = (u32)lo;
    cand_v[k] = row[j - off[lo]];
  }
}

// flag[j] = candidate j passes the label test and every constraint except
// its generator.
__global__ void filter_cands(const StepParams p, u64 n, const u32 *__restrict__ cand_t, const u32 *__restrict__ cand_v,
                             const uint8_t *__restrict__ which, u32 *__restrict__ flag) {
  for (u64 j = (u64)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (u64)gridDim.x * blockDim.x) {
    u32 y = cand_v[j];
    bool ok = p.want_label < 0 || p.vlabel[y] == (uint8_t)p.want_label;
    u32 skip = which ? which[cand_t[j]] : 0xffu;
    for (u32 k = 0; k < p.nc && ok; k++) {
      if (k == skip) continue;
      u32 x = p.c[k].col ? p.c[k].col[cand_t[j]] : y;
      const u32 *row;
      u32 l;
      const u64 *bits = lookup(p.c[k].rows, x, &row, &l);
      ok = member(row, l, bits, y);
    }
    flag[j] = ok ? 1u : 0u;
  }
}

__global__ void compact_cands(u64 n, const u32 *__restrict__ flag, const u64 *__restrict__ pos,
                              const u32 *__restrict__ cand_t, const u32 *__restrict__ cand_v, u32 ncols,
                              const ColPtrs cols) {
  for (u64 j = (u64)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (u64)gridDim.x * blockDim.x) {
    if (!flag[j]) continue;
    u64 o = pos[j];
    u32 t = cand_t ? cand_t[j] : 0;
    for (u32 c = 0; c < ncols; c++) cols.out[c][o] = cols.in[c][t];
    cols.out[ncols][o] = cand_v[j];
  }
}

// Row index of one chunk: lane i (source lanesrc[i]) is row lane_base + i.
__global__ void rows_index(const u32 *__restrict__ lanesrc, const u64 *__restrict__ lane_off, u32 n_lanes,
                           u32 lane_base, const u32 *__restrict__ dst, const u32 *__restrict__ lane_slot,
                           const u64 *__restrict__ bits, u64 bwords, u32 *__restrict__ src, u64 *__restrict__ ptr,
                           u64 *__restrict__ bptr, u32 *__restrict__ len, u32 lists_kept) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < n_lanes; i += gridDim.x * blockDim.x) {
    const u32 s = lanesrc[i];
    if (s == NO_SOURCE) continue;
    const u32 slot = lane_slot ? lane_slot[i] : NO_SOURCE;
    src[lane_base + i] = s;
    bptr[lane_base + i] = slot == NO_SOURCE ? 0ull : reinterpret_cast<u64>(bits + (u64)slot * bwords);
    if (slot == NO_SOURCE || lists_kept) {
      ptr[lane_base + i] = reinterpret_cast<u64>(dst + lane_off[i]);
      len[lane_base + i] = (u32)(lane_off[i + 1] - lane_off[i]);
    } else {
      ptr[lane_base + i] = 0;
    }
  }
}

// Vertices of label `label` as a bitset (bwords words).
__global__ void label_bits(const uint8_t *__restrict__ vlabel, u32 n, uint8_t label, u64 bwords,
                           u64 *__restrict__ out) {
  for (u64 w = (u64)blockIdx.x * blockDim.x + threadIdx.x; w < bwords; w += (u64)gridDim.x * blockDim.x) {
    u64 m = 0;
    for (u32 b = 0; b < 64; b++) {
      const u64 v = w * 64 + b;
      if (v < n && vlabel[v] == label) m |= 1ull << b;
    }
    out[w] = m;
  }
}

__global__ void widen_u32(const u32 *__restrict__ v, u64 n, u64 *__restrict__ keys) {
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) keys[i] = v[i];
}

__global__ void narrow_u64(const u64 *__restrict__ keys, u64 n, u32 *__restrict__ v) {
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x)
    v[i] = (u32)keys[i];
}

__global__ void sort_keys_from_perm(const u32 *__restrict__ col, const u32 *__restrict__ perm, u64 n,
                                    u64 *__restrict__ keys) {
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
    u32 r = perm ? perm[i] : (u32)i;
    keys[i] = ((u64)col[r] << 32) | r;
  }
}

__global__ void gather_rows(const ColPtrs cols, u32 arity, const u32 *__restrict__ perm, u64 n,
                            u32 *__restrict__ out) {
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
    u32 r = perm[i];
    for (u32 c = 0; c < arity; c++) out[i * arity + c] = cols.in[c][r];
  }
}

// Digest of tuples given as declaration-order columns (see result_info).
__global__ void digest_rows(const ColPtrs cols, u32 arity, u64 n, u64 *__restrict__ digest) {
  u64 s = 0, x = 0;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
    u64 h;
    if (arity == 1) {
      h = splitmix64((u64)cols.in[0][i]);
    } else {
      h = splitmix64(((u64)cols.in[0][i] << 32) | (u64)cols.in[1][i]);
      for (u32 c = 2; c < arity; c++) h = splitmix64(h ^ (u64)cols.in[c][i]);
    }
    s += h;
    x ^= h;
  }
  s = warp_sum(s);
  x = warp_xor(x);
  if (lane_id() == 0 && (s | x)) {
    atomicAdd(&digest[0], s);
    atomicXor(&digest[1], x);
  }
}

// Count-only binding of the last variable, fused: the tuples' work is cut
// into items (numbered by the exclusive scan coff of the tuples' item
// counts) and a warp takes one item at a time, looks up the rows of the
// tuple's constraints once, and counts and digests the tuples that extend it
// in place (no candidate arrays, no compaction, no second pass over the
// tuples).  An item of a tuple with a generating row is LAST_CHUNK of that
// row's candidates, each tested against the vertex label and every other
// constraint (bitset or binary search); an item of a DENSE tuple (all rows
// bitsets) is DENSE_WORDS words of the AND of the rows' bitsets and the
// label's, whose set bits are the new values.  The tuples are distinct
// because every bound value of a partial tuple is, and every candidate of a
// sorted row or bit of a bitset.
constexpr u32 LAST_CHUNK = 256;
constexpr u32 DENSE_WORDS = 2048;

constexpr u64 ITEM_BLOCK = 16;  // consecutive items a warp takes at a time

struct LastParams {
  StepParams p;
  unsigned long long *cursor;    // next unclaimed item (zero at launch)
  const uint8_t *which;          // generating constraint per tuple, or DENSE
  const u32 *cnt;                // its row length
  const u64 *coff;               // exclusive scan of the tuples' item counts
  u64 nT, items;
  u32 arity;                     // variables of the query
  u32 newpos;                    // declaration position of the variable being bound
  const u32 *dcol[RPQ_MAX_VARS]; // declaration-order columns of the bound variables (nullptr: the new one)
  u64 *acc;                      // [0] digest sum, [1] digest xor, [5] count
};

constexpr int CL_THREADS = 256;
constexpr int CL_WARPS = CL_THREADS / 32;

// Per-warp state of an item: the rows of the tuple's constraints and the
// tuple's bound values (declaration order).
struct LastWarp {
  const u32 *row[MAXC];
  const u64 *bits[MAXC];
  u32 len[MAXC];
  u32 vals[RPQ_MAX_VARS];
};

// Digest hash of the tuple (bound values with z at position newpos), given
// pre = the fold over positions 0 .. newpos - 1 when newpos >= 2 (see
// result_info).
__device__ __forceinline__ u64 last_hash(const LastParams &lp, const LastWarp &sw, u64 pre, u32 z) {
  if (lp.newpos >= 2 && lp.newpos + 1 == lp.arity) return splitmix64(pre ^ (u64)z);  // the common case
  if (lp.arity == 1) return splitmix64((u64)z);
  u64 h;
  u32 v;
  if (lp.newpos >= 2) {
    h = splitmix64(pre ^ (u64)z);
    v = lp.newpos + 1;
  } else {
    const u32 a0 = lp.newpos == 0 ? z : sw.vals[0], a1 = lp.newpos == 1 ? z : sw.vals[1];
    h = splitmix64(((u64)a0 << 32) | (u64)a1);
    v = 2;
  }
  for (; v < lp.arity; v++) h = splitmix64(h ^ (u64)sw.vals[v]);
  return h;
}

__global__ void __launch_bounds__(CL_THREADS) count_last_kernel(const LastParams lp) {
  __shared__ LastWarp s_warp[CL_WARPS];
  const StepParams &p = lp.p;
  LastWarp &sw = s_warp[threadIdx.x >> 5];
  const u32 lane = lane_id();
  u64 cnt = 0, hs = 0, hx = 0;
  // Warps take blocks of ITEM_BLOCK consecutive items from a cursor: the
  // tuple of a block's first item is found by one binary search over coff,
  // and a tuple's rows are looked up once for all its items in the block.
  u64 i = 0, cur_beg = 0, nxt_beg = 0, t = 0, te = 0;
  u32 gen = 0;
  u64 pre = 0;
  for (;;) {
    if (t == te) {  // next block
      u64 tb = 0;
      if (lane == 0) tb = atomicAdd(lp.cursor, (unsigned long long)ITEM_BLOCK);
      tb = __shfl_sync(FULL_MASK, tb, 0);
      if (tb >= lp.items) break;
      t = tb;
      te = min(lp.items, tb + ITEM_BLOCK);
      // the tuple of item t: the largest i with coff[i] <= t
      u64 lo = 0, hi = lp.nT;
      while (hi - lo > 1) {
        const u64 mid = (lo + hi) >> 1;
        if (lp.coff[mid] <= t)
          lo = mid;
        else
          hi = mid;
      }
      i = lo;
      cur_beg = lp.coff[i];
      nxt_beg = i + 1 < lp.nT ? lp.coff[i + 1] : ~0ull;
      gen = 0xFFFFFFFFu;  // rows not looked up yet
    }
    if (t >= nxt_beg) {  // the next tuple with items (tuples without items are skipped)
      do {
        ++i;
        cur_beg = nxt_beg;
        nxt_beg = i + 1 < lp.nT ? lp.coff[i + 1] : ~0ull;
      } while (t >= nxt_beg);
      gen = 0xFFFFFFFFu;
    }
    if (gen == 0xFFFFFFFFu) {
      gen = lp.which[i];
      __syncwarp();  // the previous tuple's readers are done
      // rows of the tuple's constraints (lane k looks up constraint k), bound values
      if (lane < p.nc) sw.bits[lane] = lookup(p.c[lane].rows, p.c[lane].col[i], &sw.row[lane], &sw.len[lane]);
      if (lane < lp.arity) sw.vals[lane] = lp.dcol[lane] ? lp.dcol[lane][i] : 0u;
      __syncwarp();
      pre = 0;
      if (lp.newpos >= 2) {
        pre = splitmix64(((u64)sw.vals[0] << 32) | (u64)sw.vals[1]);
        for (u32 v = 2; v < lp.newpos; v++) pre = splitmix64(pre ^ (u64)sw.vals[v]);
      }
    }
    const u32 c = (u32)(t - cur_beg);
    t++;
    if (gen == DENSE) {
      // words w0 + lane + 32 j of the AND, four per round; a lane walks the
      // set bits of its four words in one loop, so that lanes wait for the
      // largest four-word count rather than the largest one-word count
      const u64 *b0 = sw.bits[0], *b1 = p.nc > 1 ? sw.bits[1] : nullptr;
      const u64 w0 = (u64)c * DENSE_WORDS, w1 = min(p.bwords, w0 + DENSE_WORDS);
      for (u64 wb = w0; wb < w1; wb += 128) {
        u64 m[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
          const u64 w = wb + lane + 32 * j;
          u64 x = 0;
          if (w < w1) {
            x = p.lbits ? p.lbits[w] : ~0ull;
            x &= b0[w];
            if (b1) x &= b1[w];
            for (u32 k = 2; k < p.nc; k++) x &= sw.bits[k][w];
          }
          m[j] = x;
        }
        // the eight 32-bit halves in vertex order: half k covers vertices
        // base0 + (k / 2) * 2048 + (k % 2) * 32 ..
        u32 hm[7];
#pragma unroll
        for (int k = 0; k < 7; k++) hm[k] = (u32)(m[(k + 1) >> 1] >> (((k + 1) & 1) * 32));
        u32 cur = (u32)m[0], k = 0, c32 = 0;
        const u32 base0 = (u32)((wb + lane) * 64);
        for (;;) {
          while (!cur && k < 7) {  // next half of the four words
            cur = hm[0];
#pragma unroll
            for (int r = 0; r < 6; r++) hm[r] = hm[r + 1];
            k++;
          }
          if (!cur) break;
          const u32 z = base0 + (k >> 1) * 2048 + (k & 1) * 32 + (__ffs(cur) - 1);
          const u64 h = last_hash(lp, sw, pre, z);
          cur &= cur - 1;
          c32++;
          hs += h;
          hx ^= h;
        }
        cnt += c32;
      }
      continue;
    }
    const u32 *grow = sw.row[gen];
    const u32 end = min(sw.len[gen], (c + 1) * LAST_CHUNK);
    for (u32 j = c * LAST_CHUNK + lane; j < end; j += 32) {
      const u32 z = grow[j];
      bool ok = p.want_label < 0 || p.vlabel[z] == (uint8_t)p.want_label;
      for (u32 k = 0; k < p.nc && ok; k++)
        if (k != gen) ok = member(sw.row[k], sw.len[k], sw.bits[k], z);
      if (!ok) continue;
      const u64 h = last_hash(lp, sw, pre, z);
      cnt++;
      hs += h;
      hx ^= h;
    }
  }
  cnt = warp_sum(cnt);
  hs = warp_sum(hs);
  hx = warp_xor(hx);
  if (lane == 0 && cnt) {
    atomicAdd(&lp.acc[5], cnt);
    atomicAdd(&lp.acc[0], hs);
    atomicXor(&lp.acc[1], hx);
  }
}

// Items per tuple of the fused last step.
__global__ void chunk_counts(const u32 *__restrict__ cnt, const uint8_t *__restrict__ which, u64 n, u64 bwords,
                             u32 *__restrict__ out) {
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x)
    out[i] = which[i] == DENSE ? (u32)((bwords + DENSE_WORDS - 1) / DENSE_WORDS)
                               : (cnt[i] + LAST_CHUNK - 1) / LAST_CHUNK;
}

unsigned grid1(u64 n) {
  u64 b = (n + 255) / 256;
  if (b > 152ull * 32) b = 152ull * 32;
  return (unsigned)(b ? b : 1);
}

// Device buffer owned through the context's budget.
template <typename T>
struct Buf {
  rpq_ctx *ctx = nullptr;
  T *p = nullptr;
  uint64_t n = 0;
  int alloc(rpq_ctx *c, uint64_t count) {
    release();
    ctx = c;
    n = count;
    return ctx_alloc(c, (void **)&p, std::max<uint64_t>(count, 1) * sizeof(T));
  }
  void release() {
    if (p) ctx_free(ctx, p, std::max<uint64_t>(n, 1) * sizeof(T));
    p = nullptr;
    n = 0;
  }
  ~Buf() { release(); }
};

// Rows of one atom: an index over the values (sorted) pointing into the
// chunks the traversals wrote, which the rows own.
struct OwnedRows {
  rpq_ctx *ctx = nullptr;
  Buf<u32> src, len;
  Buf<u64> ptr, bptr;
  std::vector<RowChunk> chunks;
  u32 ns = 0;
  DevRows view() const { return DevRows{src.p, ptr.p, bptr.p, len.p, ns}; }
  ~OwnedRows() {
    for (auto &c : chunks) free_row_chunk(ctx, c);
  }
};

struct Table {
  std::vector<Buf<u32>> cols;  // binding order
  uint64_t n = 0;
};

struct Engine {
  rpq_ctx *ctx;
  const rpq_graph *g;
  const DevGraph &dg;
  cudaStream_t st;
  uint32_t n_vars;
  const int32_t *var_label;
  const crpq_atom *atoms;
  bool materialize;
  std::vector<int> order, pos;
  struct C {
    uint32_t atom;
    int bound_pos;  // -1: self-loop on the variable being bound
    bool reverse;
  };
  std::vector<std::vector<C>> cons;
  rpq_stats stats;
  uint64_t count = 0, dsum = 0, dxor = 0;
  Buf<u64> small;                       // digest accumulators, counters
  std::vector<Table> batch_out;         // complete tables of the current batch
  std::vector<std::pair<u32 *, uint64_t>> out_chunks;  // sorted row-major batches
  double t_rows = 0, t_gen = 0, t_join = 0;  // host seconds per phase (trace)
  Buf<u64> lbits;        // vertices of label lbits_label as a bitset
  int lbits_label = -1;

  Engine(rpq_ctx *c, const rpq_graph *gr) : ctx(c), g(gr), dg(graph_dev(gr)), st(ctx_stream(c)) {
    std::memset(&stats, 0, sizeof(stats));
  }

  int cuda(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return RPQ_OK;
    return ctx_error(ctx, RPQ_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  }

  int label_of(uint32_t var) const { return var_label ? var_label[var] : -1; }

  // Distinct values of a device column, ascending, on the host.
  int distinct(const u32 *col, uint64_t n, std::vector<uint32_t> *out) {
    out->clear();
    if (n == 0) return RPQ_OK;
    Buf<u64> a, b;
    int rc;
    if ((rc = a.alloc(ctx, n)) || (rc = b.alloc(ctx, n))) return rc;
    widen_u32<<<grid1(n), 256, 0, st>>>(col, n, a.p);
    if ((rc = cuda(cudaGetLastError(), "widen_u32"))) return rc;
    u64 *pa = a.p, *pb = b.p;
    if ((rc = cuda(sort_keys_u64(&pa, &pb, n, 0, 32, st), "sort"))) return rc;
    if ((rc = cuda(unique_keys_u64(pa, n, pb, small.p + 2, st), "unique"))) return rc;
    u64 k = 0;
    if ((rc = cuda(cudaMemcpyAsync(&k, small.p + 2, 8, cudaMemcpyDeviceToHost, st), "copy"))) return rc;
    if ((rc = cuda(cudaStreamSynchronize(st), "sync"))) return rc;
    std::vector<u64> tmp(k);
    if (k && (rc = cuda(cudaMemcpyAsync(tmp.data(), pb, k * 8, cudaMemcpyDeviceToHost, st), "copy"))) return rc;
    if ((rc = cuda(cudaStreamSynchronize(st), "sync"))) return rc;
    out->resize(k);
    for (u64 i = 0; i < k; i++) (*out)[i] = (uint32_t)tmp[i];
    return RPQ_OK;
  }

  // Rows of atom `a` for the given sorted distinct values.  Rows of at least
  // crpq_bitset_frac * n destinations also come out as bitsets; with
  // `fused` (a count-only last step) such rows are kept as bitsets only.
  int rows_for(uint32_t a, bool reverse, std::vector<uint32_t> &vals, OwnedRows *r, bool fused) {
    const double frac = ctx_crpq_bitset_frac(ctx);
    RowBitsReq req;
    req.min_len = std::max<uint64_t>(1, (uint64_t)std::ceil(frac * dg.n));
    req.keep_lists = !fused;
    const double t0 = host_seconds();
    r->ctx = ctx;
    int rc = rpq_rows_for_sources(ctx, g, atoms[a].q, vals, reverse, &r->chunks, &stats, nullptr, nullptr,
                                  frac > 1.0 ? nullptr : &req);
    const double t1 = host_seconds();
    t_rows += t1 - t0;
    r->ns = (u32)vals.size();
    if (!rc && ((rc = r->src.alloc(ctx, r->ns)) || (rc = r->ptr.alloc(ctx, r->ns)) ||
                (rc = r->bptr.alloc(ctx, r->ns)) || (rc = r->len.alloc(ctx, r->ns)))) {
    }
    if (!rc && r->ns) {
      // a value without a lane (no edge out of its start state, or an empty
      // language) has no row: lookups of it find none
      cudaMemsetAsync(r->len.p, 0, (uint64_t)r->ns * 4, st);
      cudaMemsetAsync(r->ptr.p, 0, (uint64_t)r->ns * 8, st);
      cudaMemsetAsync(r->bptr.p, 0, (uint64_t)r->ns * 8, st);
      cudaMemsetAsync(r->src.p, 0xff, (uint64_t)r->ns * 4, st);
    }
    uint32_t lane_base = 0;
    uint64_t n_bits = 0;
    for (auto &c : r->chunks) {
      if (!rc) {
        rows_index<<<grid1(c.n_lanes), 256, 0, st>>>(c.lanesrc, c.lane_off, c.n_lanes, lane_base, c.dst,
                                                     c.lane_slot, c.bits, c.bwords, r->src.p, r->ptr.p, r->bptr.p,
                                                     r->len.p, c.lists_kept ? 1u : 0u);
        rc = cuda(cudaGetLastError(), "rows_index");
        stats.launches += 1;
      }
      lane_base += c.n_lanes;
      n_bits += c.n_bits;
    }
    if (ctx_trace(ctx)) {
      uint64_t listed = 0;
      for (auto &c : r->chunks) listed += c.rows;
      std::fprintf(stderr, "[rpq trace] crpq rows=%u listed=%llu bitsets=%llu (%.1f MB) %s\n", r->ns,
                   (unsigned long long)listed, (unsigned long long)n_bits,
                   n_bits * (((uint64_t)dg.n + 255) / 256 * 4) * 8 / 1e6, fused ? "bitsets only" : "lists kept");
    }
    return rc;
  }

  // Vertices of label `label` as a bitset of bwords words (kept per engine).
  int label_bitset(int label, uint64_t bwords, const u64 **out) {
    int rc;
    if (lbits_label != label) {
      if ((rc = lbits.alloc(ctx, bwords))) return rc;
      label_bits<<<grid1(bwords), 256, 0, st>>>(dg.vlabel, dg.n, (uint8_t)label, bwords, lbits.p);
      if ((rc = cuda(cudaGetLastError(), "label_bits"))) return rc;
      stats.launches += 1;
      lbits_label = label;
    }
    *out = lbits.p;
    return RPQ_OK;
  }

  // Binds variable order[k] from the candidates (cand_t, cand_v) of table T
  // (cand_t == nullptr when T has no columns), filtering with `p`.
  int bind(int k, Table &T, const u32 *cand_t, const u32 *cand_v, uint64_t nc, StepParams &p,
           const uint8_t *which) {
    if (nc == 0) return RPQ_OK;
    Buf<u32> flag;
    Buf<u64> posb, tmp;
    int rc;
    if ((rc = flag.alloc(ctx, nc)) || (rc = posb.alloc(ctx, nc)) || (rc = tmp.alloc(ctx, scan_tmp_words(nc))))
      return rc;
    filter_cands<<<grid1(nc), 256, 0, st>>>(p, nc, cand_t, cand_v, which, flag.p);
    if ((rc = cuda(cudaGetLastError(), "filter_cands"))) return rc;
    if ((rc = cuda(exclusive_scan_u32_to_u64(flag.p, posb.p, nc, small.p + 3, tmp.p, st), "scan"))) return rc;
    u64 kept = 0;
    if ((rc = cuda(cudaMemcpyAsync(&kept, small.p + 3, 8, cudaMemcpyDeviceToHost, st), "copy"))) return rc;
    if ((rc = cuda(cudaStreamSynchronize(st), "sync"))) return rc;
    stats.launches += 3;
    if (kept == 0) return RPQ_OK;
    Table N;
    N.n = kept;
    N.cols.resize(k + 1);
    ColPtrs cp;
    std::memset(&cp, 0, sizeof(cp));
    for (int c = 0; c <= k; c++) {
      if ((rc = N.cols[c].alloc(ctx, kept))) return rc;
      cp.out[c] = N.cols[c].p;
      if (c < k) cp.in[c] = T.cols[c].p;
    }
    compact_cands<<<grid1(nc), 256, 0, st>>>(nc, flag.p, posb.p, cand_t, cand_v, (u32)k, cp);
    if ((rc = cuda(cudaGetLastError(), "compact_cands"))) return rc;
    stats.launches += 1;
    flag.release();
    posb.release();
    tmp.release();
    return extend(k + 1, N);
  }

  // Fills p.c for the constraints of position k; self-loop rows come from
  // the candidate values.  fused: the count-only last step.
  int prepare(int k, Table &T, const u32 *cand_v, uint64_t nc, std::vector<OwnedRows> &rows, StepParams &p,
              bool self_only, bool fused) {
    std::memset(&p, 0, sizeof(p));
    p.want_label = label_of((uint32_t)order[k]);
    p.vlabel = dg.vlabel;
    p.fused = fused ? 1u : 0u;
    p.bwords = ((uint64_t)dg.n + 255) / 256 * 4;
    rows.resize(cons[k].size());
    int rc;
    for (size_t i = 0; i < cons[k].size(); i++) {
      const C &c = cons[k][i];
      if ((c.bound_pos < 0) != self_only) continue;
      std::vector<uint32_t> vals;
      if (c.bound_pos < 0)
        rc = distinct(cand_v, nc, &vals);
      else
        rc = distinct(T.cols[c.bound_pos].p, T.n, &vals);
      if (rc) return rc;
      if ((rc = rows_for(c.atom, c.reverse, vals, &rows[i], fused))) return rc;
    }
    if (fused && p.want_label >= 0 && (rc = label_bitset(p.want_label, p.bwords, &p.lbits))) return rc;
    p.nc = (u32)cons[k].size();
    for (size_t i = 0; i < cons[k].size(); i++) {
      p.c[i].rows = rows[i].view();
      p.c[i].col = cons[k][i].bound_pos < 0 ? nullptr : T.cols[cons[k][i].bound_pos].p;
      if (cons[k][i].bound_pos >= 0) p.gen_mask |= 1u << i;
    }
    return RPQ_OK;
  }

  int extend(int k, Table &T) {
    if (T.n == 0) return RPQ_OK;
    if (k == (int)n_vars) return emit(T);
    bool has_self = false;
    for (auto &c : cons[k]) has_self |= c.bound_pos < 0;
    const bool fused = k == (int)n_vars - 1 && !materialize && !has_self;
    std::vector<OwnedRows> rows;
    StepParams p;
    int rc = prepare(k, T, nullptr, 0, rows, p, false, fused);
    if (rc) return rc;
    Buf<u32> cnt;
    Buf<uint8_t> which;
    Buf<u64> off, tmp;
    if ((rc = cnt.alloc(ctx, T.n)) || (rc = which.alloc(ctx, T.n)) || (rc = off.alloc(ctx, T.n + 1)) ||
        (rc = tmp.alloc(ctx, scan_tmp_words(T.n + 1))))
      return rc;
    const double t0 = host_seconds();
    choose_gen<<<grid1(T.n), 256, 0, st>>>(p, T.n, cnt.p, which.p);
    if ((rc = cuda(cudaGetLastError(), "choose_gen"))) return rc;
    if ((rc = cuda(exclusive_scan_u32_to_u64(cnt.p, off.p, T.n, small.p + 4, tmp.p, st), "scan"))) return rc;
    u64 total = 0;
    if ((rc = cuda(cudaMemcpyAsync(&total, small.p + 4, 8, cudaMemcpyDeviceToHost, st), "copy"))) return rc;
    if ((rc = cuda(cudaMemcpyAsync(off.p + T.n, small.p + 4, 8, cudaMemcpyDeviceToDevice, st), "copy"))) return rc;
    if ((rc = cuda(cudaStreamSynchronize(st), "sync"))) return rc;
    stats.launches += 2;
    t_gen += host_seconds() - t0;
    if (ctx_trace(ctx))
      std::fprintf(stderr, "[rpq trace] crpq bind k=%d tuples=%llu candidates=%llu\n", k, (unsigned long long)T.n,
                   (unsigned long long)total);
    if (fused) return count_last(k, T, p, cnt.p, which.p);
    for (u64 c0 = 0; c0 < total; c0 += CAND_CAP) {
      u64 nc = std::min<u64>(CAND_CAP, total - c0);
      Buf<u32> ct, cv;
      if ((rc = ct.alloc(ctx, nc)) || (rc = cv.alloc(ctx, nc))) return rc;
      expand_cands<<<grid1(nc), 256, 0, st>>>(p, T.n, off.p, which.p, c0, nc, ct.p, cv.p);
      if ((rc = cuda(cudaGetLastError(), "expand_cands"))) return rc;
      stats.launches += 1;
      // self-loop constraints need the candidate values
      std::vector<OwnedRows> self_rows;
      StepParams ps = p;
      if (has_self) {
        StepParams tmpp;
        if ((rc = prepare(k, T, cv.p, nc, self_rows, tmpp, true, false))) return rc;
        for (size_t i = 0; i < cons[k].size(); i++)
          if (cons[k][i].bound_pos < 0) ps.c[i].rows = self_rows[i].view();
      }
      if ((rc = bind(k, T, ct.p, cv.p, nc, ps, which.p))) return rc;
    }
    return RPQ_OK;
  }

  // The last variable of a count-only query: fused binding, count and digest.
  int count_last(int k, Table &T, const StepParams &p, const u32 *cnt, const uint8_t *which) {
    Buf<u32> nch;
    Buf<u64> coff, tmp;
    int rc;
    if ((rc = nch.alloc(ctx, T.n)) || (rc = coff.alloc(ctx, T.n + 1)) ||
        (rc = tmp.alloc(ctx, scan_tmp_words(T.n + 1))))
      return rc;
    chunk_counts<<<grid1(T.n), 256, 0, st>>>(cnt, which, T.n, p.bwords, nch.p);
    if ((rc = cuda(cudaGetLastError(), "chunk_counts"))) return rc;
    if ((rc = cuda(exclusive_scan_u32_to_u64(nch.p, coff.p, T.n, small.p + 4, tmp.p, st), "scan"))) return rc;
    u64 items = 0, got = 0;
    if ((rc = cuda(cudaMemcpyAsync(&items, small.p + 4, 8, cudaMemcpyDeviceToHost, st), "copy")) ||
        (rc = cuda(cudaMemsetAsync(small.p + 5, 0, 16, st), "memset")) || (rc = cuda(cudaStreamSynchronize(st), "sync")))
      return rc;
    LastParams lp;
    std::memset(&lp, 0, sizeof(lp));
    lp.p = p;
    lp.which = which;
    lp.cnt = cnt;
    lp.coff = coff.p;
    lp.nT = T.n;
    lp.items = items;
    lp.arity = n_vars;
    lp.newpos = (u32)order[k];
    for (uint32_t v = 0; v < n_vars; v++) lp.dcol[v] = pos[v] < k ? T.cols[pos[v]].p : nullptr;
    lp.acc = small.p;
    lp.cursor = reinterpret_cast<unsigned long long *>(small.p + 6);
    const double t0 = host_seconds();
    if (items) {
      const u64 warps = std::min<u64>(items, 152ull * 64);
      count_last_kernel<<<(unsigned)((warps * 32 + CL_THREADS - 1) / CL_THREADS), CL_THREADS, 0, st>>>(lp);
      if ((rc = cuda(cudaGetLastError(), "count_last"))) return rc;
    }
    if ((rc = cuda(cudaMemcpyAsync(&got, small.p + 5, 8, cudaMemcpyDeviceToHost, st), "copy")) ||
        (rc = cuda(cudaStreamSynchronize(st), "sync")))
      return rc;
    stats.launches += 3;
    t_join += host_seconds() - t0;
    count += got;
    return RPQ_OK;
  }

  int emit(Table &T) {
    ColPtrs cp;
    std::memset(&cp, 0, sizeof(cp));
    for (uint32_t v = 0; v < n_vars; v++) cp.in[v] = T.cols[pos[v]].p;
    digest_rows<<<grid1(T.n), 256, 0, st>>>(cp, n_vars, T.n, small.p);
    int rc = cuda(cudaGetLastError(), "digest_rows");
    if (rc) return rc;
    stats.launches += 1;
    count += T.n;
    if (materialize) batch_out.push_back(std::move(T));
    return RPQ_OK;
  }

  // Sorts the complete tuples of a batch and appends them row-major.
  int flush_batch() {
    uint64_t n = 0;
    for (auto &t : batch_out) n += t.n;
    if (n == 0 || !materialize) {
      batch_out.clear();
      return RPQ_OK;
    }
    if (n >= (1ull << 32)) return ctx_error(ctx, RPQ_ERR_OUT_OF_BUDGET, "more than 2^32 tuples in one batch");
    int rc;
    // concatenate declaration-order columns
    std::vector<Buf<u32>> cols(n_vars);
    for (uint32_t v = 0; v < n_vars; v++) {
      if ((rc = cols[v].alloc(ctx, n))) return rc;
      uint64_t o = 0;
      for (auto &t : batch_out) {
        if ((rc = cuda(cudaMemcpyAsync(cols[v].p + o, t.cols[pos[v]].p, t.n * 4, cudaMemcpyDeviceToDevice, st),
                       "copy")))
          return rc;
        o += t.n;
      }
    }
    batch_out.clear();
    // LSD over columns: last column first, each pass stable on the high word
    Buf<u64> ka, kb;
    Buf<u32> perm;
    if ((rc = ka.alloc(ctx, n)) || (rc = kb.alloc(ctx, n)) || (rc = perm.alloc(ctx, n))) return rc;
    for (int v = (int)n_vars - 1; v >= 0; v--) {
      sort_keys_from_perm<<<grid1(n), 256, 0, st>>>(cols[v].p, v == (int)n_vars - 1 ? nullptr : perm.p, n, ka.p);
      if ((rc = cuda(cudaGetLastError(), "sort_keys"))) return rc;
      u64 *pa = ka.p, *pb = kb.p;
      if ((rc = cuda(sort_keys_u64(&pa, &pb, n, 32, 64, st), "sort"))) return rc;
      narrow_u64<<<grid1(n), 256, 0, st>>>(pa, n, perm.p);
      if ((rc = cuda(cudaGetLastError(), "narrow"))) return rc;
      stats.launches += 2;
    }
    u32 *rowsp = nullptr;
    if ((rc = ctx_alloc(ctx, (void **)&rowsp, n * n_vars * 4))) return rc;
    ColPtrs cp;
    std::memset(&cp, 0, sizeof(cp));
    for (uint32_t v = 0; v < n_vars; v++) cp.in[v] = cols[v].p;
    gather_rows<<<grid1(n), 256, 0, st>>>(cp, n_vars, perm.p, n, rowsp);
    if ((rc = cuda(cudaGetLastError(), "gather_rows"))) {
      ctx_free(ctx, rowsp, n * n_vars * 4);
      return rc;
    }
    stats.launches += 1;
    out_chunks.push_back({rowsp, n});
    return RPQ_OK;
  }

  int plan(const crpq_atom *at, uint32_t n_atoms) {
    order.assign(1, 0);
    pos.assign(n_vars, -1);
    pos[0] = 0;
    while (order.size() < n_vars) {
      int best = -1, best_score = -1;
      for (uint32_t v = 0; v < n_vars; v++) {
        if (pos[v] >= 0) continue;
        int score = 0;
        for (uint32_t a = 0; a < n_atoms; a++) {
          if (at[a].y == v && at[a].x != v && pos[at[a].x] >= 0) score += 3;  // forward
          if (at[a].x == v && at[a].y != v && pos[at[a].y] >= 0) score += 2;  // reverse
        }
        if (score > best_score) {
          best = (int)v;
          best_score = score;
        }
      }
      if (best_score <= 0) return ctx_error(ctx, RPQ_ERR_INVALID_ARG, "the atoms do not connect all variables");
      pos[best] = (int)order.size();
      order.push_back(best);
    }
    cons.assign(n_vars, {});
    for (uint32_t a = 0; a < n_atoms; a++) {
      int px = pos[at[a].x], py = pos[at[a].y];
      if (at[a].x == at[a].y)
        cons[px].push_back(C{a, -1, false});
      else if (py > px)
        cons[py].push_back(C{a, px, false});
      else
        cons[px].push_back(C{a, py, true});
      if (cons[std::max(px, py)].size() > (size_t)MAXC) return ctx_error(ctx, RPQ_ERR_TOO_COMPLEX, "too many atoms");
    }
    for (int k = 1; k < (int)n_vars; k++) {
      bool gen = false;
      for (auto &c : cons[k]) gen |= c.bound_pos >= 0;
      if (!gen) return ctx_error(ctx, RPQ_ERR_INVALID_ARG, "the atoms do not connect all variables");
    }
    return RPQ_OK;
  }
};

}  // namespace

int crpq_eval(rpq_ctx *ctx, const rpq_graph *g, uint32_t n_vars, const int32_t *var_label, const crpq_atom *atoms,
              uint32_t n_atoms, const uint32_t *restrict0, uint32_t n_restrict0, uint32_t flags, rpq_result **out) {
  if (n_vars == 0 || n_vars > RPQ_MAX_VARS) return ctx_error(ctx, RPQ_ERR_INVALID_ARG, "n_vars out of range");
  if (n_atoms == 0 || n_atoms > RPQ_MAX_ATOMS) return ctx_error(ctx, RPQ_ERR_INVALID_ARG, "n_atoms out of range");
  if (flags & (RPQ_REVERSE | RPQ_FORCE_PUSH | RPQ_FORCE_PULL))
    return ctx_error(ctx, RPQ_ERR_INVALID_ARG, "run_crpq takes RPQ_MATERIALIZE or RPQ_COUNT_ONLY only");
  const DevGraph &dg = graph_dev(g);
  std::vector<char> used(n_vars, 0);
  for (uint32_t a = 0; a < n_atoms; a++) {
    if (atoms[a].x >= n_vars || atoms[a].y >= n_vars || !atoms[a].q)
      return ctx_error(ctx, RPQ_ERR_INVALID_ARG, "bad atom");
    used[atoms[a].x] = used[atoms[a].y] = 1;
  }
  for (uint32_t v = 0; v < n_vars; v++) {
    if (!used[v]) return ctx_error(ctx, RPQ_ERR_INVALID_ARG, "a variable occurs in no atom");
    if (var_label && var_label[v] >= 0 && dg.vlabel_host.empty())
      return ctx_error(ctx, RPQ_ERR_INVALID_ARG, "vertex label constraint on a graph without vertex labels");
  }
  Engine E(ctx, g);
  E.n_vars = n_vars;
  E.var_label = var_label;
  E.atoms = atoms;
  E.materialize = (flags & RPQ_MATERIALIZE) != 0;
  int rc = E.plan(atoms, n_atoms);
  if (rc) return rc;
  for (uint32_t k = 0; k < n_vars; k++)
    for (auto &c : E.cons[k])
      if (c.reverse && !query_host(atoms[c.atom].q).has_rev)
        return ctx_error(ctx, RPQ_ERR_TOO_COMPLEX, "an atom needs its reversed language, which is too large");
  if ((rc = E.small.alloc(ctx, 8))) return rc;
  cudaStream_t st = ctx_stream(ctx);
  cudaMemsetAsync(E.small.p, 0, 64, st);

  // values of variable 0
  std::vector<uint32_t> first;
  if (restrict0) {
    first.assign(restrict0, restrict0 + n_restrict0);
    for (uint32_t v : first)
      if (v >= dg.n) return ctx_error(ctx, RPQ_ERR_INVALID_ARG, "restricted vertex out of range");
    std::sort(first.begin(), first.end());
    first.erase(std::unique(first.begin(), first.end()), first.end());
  } else {
    first.resize(dg.n);
    std::iota(first.begin(), first.end(), 0u);
  }
  if (E.label_of(0) >= 0) {
    std::vector<uint32_t> keep;
    for (uint32_t v : first)
      if (dg.vlabel_host[v] == (uint8_t)E.label_of(0)) keep.push_back(v);
    first.swap(keep);
  }

  for (size_t b0 = 0; b0 < first.size() && rc == RPQ_OK; b0 += BATCH0) {
    if (ctx_cancelled(ctx)) {
      rc = ctx_error(ctx, RPQ_ERR_CANCELLED, "cancelled");
      break;
    }
    uint64_t nb = std::min<size_t>(BATCH0, first.size() - b0);
    Buf<u32> vals;
    if ((rc = vals.alloc(ctx, nb))) break;
    if ((rc = E.cuda(cudaMemcpyAsync(vals.p, first.data() + b0, nb * 4, cudaMemcpyHostToDevice, st), "copy"))) break;
    Table T0;  // no columns yet
    std::vector<OwnedRows> rows;
    StepParams p;
    if ((rc = E.prepare(0, T0, vals.p, nb, rows, p, true, false))) break;
    if ((rc = E.bind(0, T0, nullptr, vals.p, nb, p, nullptr))) break;
    rc = E.flush_batch();
  }
  if (rc) {
    for (auto &c : E.out_chunks) ctx_free(ctx, c.first, c.second * n_vars * 4);
    return rc;
  }
  if (ctx_trace(ctx))
    std::fprintf(stderr,
                 "[rpq trace] crpq rows %.1f ms generators %.1f ms count_last %.1f ms\n", E.t_rows * 1e3,
                 E.t_gen * 1e3, E.t_join * 1e3);
  // digest and final rows
  u64 dig[2] = {0, 0};
  if ((rc = E.cuda(cudaMemcpyAsync(dig, E.small.p, 16, cudaMemcpyDeviceToHost, st), "copy")) ||
      (rc = E.cuda(cudaStreamSynchronize(st), "sync"))) {
    for (auto &c : E.out_chunks) ctx_free(ctx, c.first, c.second * n_vars * 4);
    return rc;
  }
  u32 *tuples = nullptr;
  if (E.materialize && E.count) {
    if (E.out_chunks.size() == 1) {
      tuples = E.out_chunks[0].first;
    } else {
      if ((rc = ctx_alloc(ctx, (void **)&tuples, E.count * n_vars * 4))) {
        for (auto &c : E.out_chunks) ctx_free(ctx, c.first, c.second * n_vars * 4);
        return rc;
      }
      uint64_t o = 0;
      for (auto &c : E.out_chunks) {
        cudaMemcpyAsync(tuples + o * n_vars, c.first, c.second * n_vars * 4, cudaMemcpyDeviceToDevice, st);
        o += c.second;
      }
      for (auto &c : E.out_chunks) ctx_free(ctx, c.first, c.second * n_vars * 4);
    }
    cudaStreamSynchronize(st);
  } else {
    for (auto &c : E.out_chunks) ctx_free(ctx, c.first, c.second * n_vars * 4);
  }
  return make_tuple_result(ctx, n_vars, tuples, E.count, dig[0], dig[1], E.materialize, E.stats, out);
}

}  // namespace rpq
