// Result emission: visited words -> distinct (src, dst) rows in sorted order.
//
// After the search, the result set of start vertex s (Definition 1) is the
// set of v with some accepting state q such that s's lane is set in the
// visited word of (group g, state q, vertex v).  For lane group g, OR the
// accepting states' words into a K-bit result word per vertex.  A block owns
// a segment of EMIT_SEG vertices of one group and walks it in batches of
// EMIT_BATCH 32-vertex tiles.  The block loads a batch cooperatively, whole
// 32-byte sectors at a time (a vertex's K lane bits of the group are one
// contiguous run), into shared memory laid out by lane column; warp c then
// reads lane column c (32 lanes) of each tile, thread i holding the 32 lane
// bits of vertex w0 + i.
//
// Count pass: each thread adds its words into bit-sliced counters (plane k
// holds bit k of each lane's count over the thread's vertices); at the end
// each plane is transposed across the warp once and the (lane, segment)
// counts come out as popcounts.  An exclusive scan over the counts laid out
// [lane][segment] gives every row its output position directly (lanes are in
// source order, segments in vertex order).
//
// Write pass: a 32 x 32 bit transpose across the warp turns each tile around
// so that thread j holds lane j's members among the tile's 32 vertices; the
// thread appends them to a private ring in shared memory indexed by output
// position.  Whenever a row's current 128-byte-aligned chunk of the output is
// complete, the warp stores it: four rows per store instruction, eight lanes
// per row, 16 bytes per lane -- whole sectors, with only the first and last
// chunk of a row stored word by word where they are partial.  Lanes given a
// bitset (lane_slot) also store their transposed tile words there, 32 bytes
// per lane per batch of 256 vertices, and with keep_lists = 0 write no list.
#include <algorithm>

#include "device_common.cuh"
#include "rpq_internal.h"

namespace rpq {

namespace {

constexpr u32 EMIT_BATCH = 8;            // tiles per cooperative load
constexpr u32 EMIT_BV = EMIT_BATCH * 32;  // vertices per batch
constexpr u32 EMIT_RING = 64;            // ring words per row (write pass)
static_assert(EMIT_TILES % EMIT_BATCH == 0, "segments hold whole batches");

// Shared-memory words of the write pass for 2 * NW warps: the batch [2 * NW
// columns][EMIT_BV], the rings [2 * NW][32 rows][EMIT_RING], the flush slots
// [2 * NW][32].
constexpr u32 emit_write_smem_words(int nw) {
  return 2 * nw * EMIT_BV + 2 * nw * 32 * EMIT_RING + 2 * nw * 32;
}

// 32 x 32 bit transpose across a warp: on entry lane i holds row i (bit k =
// element (i, k)), on return lane j holds column j (bit i = element (i, j)).
// The recursive block transpose: stages of width 16, 8, 4, 2, 1 each swap the
// off-diagonal blocks between lanes i and i ^ s -- a shuffle, a rotate by s
// (right for the upper lane, left for the lower one) and a bit select.
__device__ __forceinline__ u32 warp_transpose32(u32 x) {
  const u32 lane = lane_id();
#pragma unroll
  for (int k = 4; k >= 0; k--) {
    const u32 s = 1u << k;
    const u32 M = k == 4 ? 0x0000FFFFu : k == 3 ? 0x00FF00FFu : k == 2 ? 0x0F0F0F0Fu : k == 1 ? 0x33333333u : 0x55555555u;
    const bool hi = (lane & s) != 0;
    const u32 y = __shfl_xor_sync(FULL_MASK, x, s);
    const u32 t = __funnelshift_r(y, y, hi ? s : 32 - s);
    const u32 keep = hi ? ~M : M;
    x = (x & keep) | (t & ~keep);
  }
  return x;
}

// Cooperative batch load, in two halves so that the next batch's loads can be
// in flight while the current one is processed.  fetch: this thread's four
// 64-bit visited words of the batch starting at vertex w_first (vertices
// w_first .. w_first + nv - 1 of group g, OR over the accepting states; zero
// past nv or n); store: put them in s_vis[column][vertex].
template <int NW>
__device__ __forceinline__ void batch_fetch(const EmitParams &p, u32 final_mask, u32 g, u32 w_first, u32 nv,
                                            u64 (&pre)[4]) {
  static_assert(EMIT_BV * NW == 4 * 64 * NW, "four words per thread");
#pragma unroll
  for (u32 r = 0; r < 4; r++) {
    const u32 k = threadIdx.x + r * (64 * NW);
    const u32 v = k / NW, h = k % NW;
    const u32 w = w_first + v;
    u64 word = 0;
    if (v < nv && w < p.n)
      for (u32 fm = final_mask; fm; fm &= fm - 1) {
        const u32 q = __ffs(fm) - 1;
        u64 x = __ldg(p.vis + (((u64)q * p.n + w) * p.G + g) * NW + h);
        if (p.final_lane) x &= __ldg(p.final_lane + ((u64)q * p.G + g) * NW + h);  // lane mode
        word |= x;
      }
    pre[r] = word;
  }
}

template <int NW>
__device__ __forceinline__ void batch_store(const u64 (&pre)[4], u32 *s_vis) {
#pragma unroll
  for (u32 r = 0; r < 4; r++) {
    const u32 k = threadIdx.x + r * (64 * NW);
    const u32 v = k / NW, h = k % NW;
    s_vis[(2 * h) * EMIT_BV + v] = (u32)pre[r];
    s_vis[(2 * h + 1) * EMIT_BV + v] = (u32)(pre[r] >> 32);
  }
}

__device__ __forceinline__ void digest_add(u64 src, u32 y, u64 &hsum, u64 &hxor) {
  const u64 h = splitmix64(src | (u64)y);
  hsum += h;
  hxor ^= h;
}

__device__ __forceinline__ void digest_flush(u64 hsum, u64 hxor, u64 *digest) {
  hsum = warp_sum(hsum);
  hxor = warp_xor(hxor);
  if (lane_id() == 0 && (hsum | hxor)) {
    atomicAdd(&digest[0], hsum);
    atomicXor(&digest[1], hxor);
  }
}

// Stores the rows whose lanes are set in R.  Row j's words [rd_j, end_j) sit
// in its ring at position mod EMIT_RING and go to base_j[rd_j .. end_j); all
// of them lie in the 32-word chunk that starts at rd_j & ~31 (base_j is
// 128-byte aligned).  Rows are taken four per round, eight lanes per row,
// four words per lane.
__device__ __forceinline__ void ring_flush(u32 R, u32 rd, u32 end, u32 *base, const u32 *ring, u32 *slots) {
  const u32 lane = lane_id();
  if (R & (1u << lane)) slots[__popc(R & lanemask_lt())] = lane;
  __syncwarp();
  const u32 n_rows = __popc(R);
  for (u32 r0 = 0; r0 < n_rows; r0 += 4) {
    const u32 idx = r0 + (lane >> 3);
    const bool act = idx < n_rows;
    const u32 j = slots[act ? idx : 0];
    const u32 rdj = __shfl_sync(FULL_MASK, rd, j);
    const u32 endj = __shfl_sync(FULL_MASK, end, j);
    u32 *bj = reinterpret_cast<u32 *>(__shfl_sync(FULL_MASK, reinterpret_cast<u64>(base), j));
    if (act) {
      const u32 piece = (rdj & ~31u) + (lane & 7) * 4;
      u32 *d = bj + piece;
      const u32 *s = ring + j * EMIT_RING + (piece & (EMIT_RING - 1));
      if (piece >= rdj && piece + 4 <= endj) {
        *reinterpret_cast<uint4 *>(d) = *reinterpret_cast<const uint4 *>(s);
      } else {
#pragma unroll
        for (u32 k = 0; k < 4; k++)
          if (piece + k >= rdj && piece + k < endj) d[k] = s[k];
      }
    }
  }
  __syncwarp();
}

}  // namespace

// Count pass: cnt[lane][segment] = the lane's members in the segment; with
// DIGEST, also the digest of those (source, y) rows (count-only results).
template <int NW, bool DIGEST>
__global__ void __launch_bounds__(64 * NW, NW == 1 ? 16 : 4) emit_count_kernel(const EmitParams p) {
  __shared__ u32 s_vis[2 * NW * EMIT_BV];
  // groups of one segment are adjacent blocks, so they read the same
  // visited lines close together in time
  const u32 g = blockIdx.x % p.G, seg = blockIdx.x / p.G;
  const u32 col = threadIdx.x >> 5, lane = lane_id();
  const u64 glane = (u64)g * (64 * NW) + col * 32 + lane;
  const u32 src = p.lanesrc[glane];
  const u32 valid_cols = __ballot_sync(FULL_MASK, src != NO_SOURCE);
  const u64 src_hi = (u64)src << 32;
  const u32 w_begin = seg * EMIT_SEG;
  const u32 n_tiles = min((u32)EMIT_TILES, (p.n - w_begin + 31) / 32);
  constexpr int CNT_PLANES = 8;  // EMIT_TILES <= 2^CNT_PLANES - 1 vertices per thread
  static_assert(EMIT_TILES < (1 << CNT_PLANES), "count planes too narrow");
  u32 planes[CNT_PLANES];
#pragma unroll
  for (int k = 0; k < CNT_PLANES; k++) planes[k] = 0;
  u32 cnt = 0;
  u64 hsum = 0, hxor = 0;
  for (u32 tb = 0; tb < n_tiles; tb += EMIT_BATCH) {
    u64 pre[4];
    batch_fetch<NW>(p, p.final_mask, g, w_begin + tb * 32, min(EMIT_BATCH, n_tiles - tb) * 32, pre);
    __syncthreads();  // the previous batch is consumed
    batch_store<NW>(pre, s_vis);
    __syncthreads();
#pragma unroll
    for (u32 t = 0; t < EMIT_BATCH; t++) {
      const u32 x = s_vis[col * EMIT_BV + t * 32 + lane] & valid_cols;  // zero past the segment's end
      if (DIGEST) {
        u32 m = warp_transpose32(x);
        cnt += __popc(m);
        const u32 w0 = w_begin + (tb + t) * 32;
        for (; m; m &= m - 1) digest_add(src_hi, w0 + __ffs(m) - 1, hsum, hxor);
      } else {
        u32 carry = x;
#pragma unroll
        for (int k = 0; k < CNT_PLANES; k++) {
          const u32 c = planes[k] & carry;
          planes[k] ^= carry;
          carry = c;
        }
      }
    }
  }
  if (!DIGEST) {
    // lane j's count = sum over planes k of 2^k * (thread bits j of plane k)
#pragma unroll
    for (int k = 0; k < CNT_PLANES; k++) cnt += (u32)__popc(warp_transpose32(planes[k])) << k;
  }
  p.cnt[glane * p.segs + seg] = cnt;
  if (DIGEST) digest_flush(hsum, hxor, p.digest);
}

// Write pass: dst[off[lane][segment] ...] = the lane's members in vertex
// order, through per-row rings in shared memory (see the head of the file).
// Positions are kept relative to base = the row's first output word rounded
// down to a 128-byte boundary; the ring slot of position x is x mod
// EMIT_RING, so a 32-word aligned chunk of the output is 32 consecutive ring
// words.
template <int NW>
__global__ void __launch_bounds__(64 * NW, NW == 1 ? 16 : 3) emit_write_kernel(const EmitParams p) {
  extern __shared__ __align__(16) u32 emit_smem[];
  constexpr u32 COLS = 2 * NW;
  const u32 g = blockIdx.x % p.G, seg = blockIdx.x / p.G;
  const u32 col = threadIdx.x >> 5, lane = lane_id();
  u32 *s_vis = emit_smem;                                           // [COLS][EMIT_BV]
  u32 *ring = emit_smem + COLS * EMIT_BV + col * 32 * EMIT_RING;    // this warp's [32][EMIT_RING]
  u32 *slots = emit_smem + COLS * EMIT_BV + COLS * 32 * EMIT_RING + col * 32;
  u32 *myring = ring + lane * EMIT_RING;
  const u64 glane = (u64)g * (64 * NW) + col * 32 + lane;
  const u32 src = p.lanesrc[glane];
  const u32 valid_cols = __ballot_sync(FULL_MASK, src != NO_SOURCE);
  const u64 pos0 = p.off[glane * p.segs + seg];
  u32 *base = p.dst + (pos0 & ~31ull);
  u32 rd = (u32)pos0 & 31u, wr = rd;  // stored / placed words of this row, relative to base
  // the lane's bitset (a 32-bit word per tile, stored 8 words = 32 bytes per
  // batch), and whether its destinations are listed as well
  u32 *bs = nullptr;
  if (p.lane_slot) {
    const u32 slot = p.lane_slot[glane];
    if (slot != NO_SOURCE) bs = reinterpret_cast<u32 *>(p.bits + (u64)slot * p.bwords);
  }
  const bool listed = !bs || p.keep_lists;
  const u32 w_begin = seg * EMIT_SEG;
  const u32 n_tiles = min((u32)EMIT_TILES, (p.n - w_begin + 31) / 32);
  u64 pre[4];
  batch_fetch<NW>(p, p.final_mask, g, w_begin, min(EMIT_BATCH, n_tiles) * 32, pre);
  for (u32 tb = 0; tb < n_tiles; tb += EMIT_BATCH) {
    const u32 nt = min(EMIT_BATCH, n_tiles - tb);
    __syncthreads();  // the previous batch is consumed
    batch_store<NW>(pre, s_vis);
    __syncthreads();
    if (tb + EMIT_BATCH < n_tiles)  // next batch in flight while this one is placed
      batch_fetch<NW>(p, p.final_mask, g, w_begin + (tb + EMIT_BATCH) * 32,
                      min(EMIT_BATCH, n_tiles - tb - EMIT_BATCH) * 32, pre);
    u32 acc[EMIT_BATCH];
#pragma unroll
    for (u32 t = 0; t < EMIT_BATCH; t++) {
      acc[t] = 0;
      if (t >= nt) continue;  // uniform across the block
      u32 m = warp_transpose32(s_vis[col * EMIT_BV + t * 32 + lane] & valid_cols);
      acc[t] = m;
      if (!listed) m = 0;
      const u32 wb = w_begin + (tb + t) * 32 - 1;
      // at most 31 words were pending, so the ring (64) holds this tile's 32
      for (; m; m &= m - 1) myring[wr++ & (EMIT_RING - 1)] = wb + __ffs(m);
      const bool full = wr > (rd | 31u);  // rd's 32-word chunk is complete
      const u32 R = __ballot_sync(FULL_MASK, full);
      if (R) {
        ring_flush(R, rd, (rd | 31u) + 1u, base, ring, slots);
        if (full) rd = (rd | 31u) + 1u;
      }
    }
    if (bs) {  // the batch's 256 vertices start on a 32-byte boundary of the bitset
      uint4 *d = reinterpret_cast<uint4 *>(bs + (w_begin + tb * 32) / 32);
      d[0] = make_uint4(acc[0], acc[1], acc[2], acc[3]);
      d[1] = make_uint4(acc[4], acc[5], acc[6], acc[7]);
    }
  }
  const u32 R = __ballot_sync(FULL_MASK, wr > rd);  // the partial last chunks
  if (R) ring_flush(R, rd, wr, base, ring, slots);
}

// Pass 1 (write = false) counts per (lane, segment), with the digest folded
// when digest = true; pass 2 (write = true, digest = false) writes the
// destinations.
cudaError_t launch_emit(int nw, bool write, bool digest, const EmitParams &p, cudaStream_t st) {
  const unsigned grid = p.segs * p.G;
  const int threads = nw == 1 ? 64 : 256;
  if (!write) {
    if (nw == 1)
      digest ? emit_count_kernel<1, true><<<grid, threads, 0, st>>>(p)
             : emit_count_kernel<1, false><<<grid, threads, 0, st>>>(p);
    else
      digest ? emit_count_kernel<4, true><<<grid, threads, 0, st>>>(p)
             : emit_count_kernel<4, false><<<grid, threads, 0, st>>>(p);
    return cudaGetLastError();
  }
  if (digest) return cudaErrorInvalidValue;  // the write pass does not fold the digest
  if (nw != 1) {
    // the NW = 4 write pass needs more than the default 48 KB; the opt-in is
    // per device, so it is repeated on every launch (an inexpensive call)
    const cudaError_t e = cudaFuncSetAttribute(emit_write_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)(emit_write_smem_words(4) * 4));
    if (e != cudaSuccess) return e;
  }
  if (nw == 1)
    emit_write_kernel<1><<<grid, threads, emit_write_smem_words(1) * 4, st>>>(p);
  else
    emit_write_kernel<4><<<grid, threads, emit_write_smem_words(4) * 4, st>>>(p);
  return cudaGetLastError();
}

// Digest of a materialized chunk's rows: block b takes lanes b, b +
// gridDim.x, ...; the rows of lane i are contiguous (dst[lane_off[i] ..
// lane_off[i + 1])) and all belong to source lanesrc[i].  The 16-byte aligned
// middle of a lane's rows is read four rows per load, two loads in flight per
// thread; the unaligned ends row by row.
__global__ void row_digest_kernel(const u32 *__restrict__ lanesrc, const u64 *__restrict__ lane_off, u32 n_lanes,
                                  const u32 *__restrict__ dst, u64 *__restrict__ digest) {
  u64 hsum = 0, hxor = 0;
  for (u32 i = blockIdx.x; i < n_lanes; i += gridDim.x) {
    const u64 src = (u64)lanesrc[i] << 32;
    const u64 b = lane_off[i], e = lane_off[i + 1];
    const u64 ab = min(e, (b + 3) & ~3ull), ae = max(ab, e & ~3ull);  // aligned middle [ab, ae)
    for (u64 r = b + threadIdx.x; r < ab; r += blockDim.x) digest_add(src, __ldcs(dst + r), hsum, hxor);
    for (u64 r = ae + threadIdx.x; r < e; r += blockDim.x) digest_add(src, __ldcs(dst + r), hsum, hxor);
    const uint4 *v = reinterpret_cast<const uint4 *>(dst + ab);
    const u64 nv = (ae - ab) / 4;
    u64 k = threadIdx.x;
    for (; k + blockDim.x < nv; k += 2ull * blockDim.x) {
      const uint4 x0 = __ldcs(v + k), x1 = __ldcs(v + k + blockDim.x);
      digest_add(src, x0.x, hsum, hxor);
      digest_add(src, x0.y, hsum, hxor);
      digest_add(src, x0.z, hsum, hxor);
      digest_add(src, x0.w, hsum, hxor);
      digest_add(src, x1.x, hsum, hxor);
      digest_add(src, x1.y, hsum, hxor);
      digest_add(src, x1.z, hsum, hxor);
      digest_add(src, x1.w, hsum, hxor);
    }
    if (k < nv) {
      const uint4 x0 = __ldcs(v + k);
      digest_add(src, x0.x, hsum, hxor);
      digest_add(src, x0.y, hsum, hxor);
      digest_add(src, x0.z, hsum, hxor);
      digest_add(src, x0.w, hsum, hxor);
    }
  }
  hsum = warp_sum(hsum);
  hxor = warp_xor(hxor);
  if (lane_id() == 0 && (hsum | hxor)) {
    atomicAdd(&digest[0], hsum);
    atomicXor(&digest[1], hxor);
  }
}

cudaError_t launch_row_digest(const uint32_t *lanesrc, const unsigned long long *lane_off, uint32_t n_lanes,
                              const uint32_t *dst, unsigned long long *digest, cudaStream_t st) {
  if (n_lanes == 0) return cudaSuccess;
  row_digest_kernel<<<n_lanes, 256, 0, st>>>(lanesrc, lane_off, n_lanes, dst, digest);
  return cudaGetLastError();
}

// Per-lane statistics (count, digest) of every lane's rows, for callers that
// need each start vertex's result summary separately.  Same tile walk as the
// count pass; the 32 x 32 tile is transposed with 32 ballots so that thread j
// holds lane 32c + j's members and folds its own digest; one set of atomics
// per lane and segment.
template <int NW>
__global__ void __launch_bounds__(64 * NW, NW == 1 ? 16 : 4) emit_lane_stats_kernel(const EmitParams p,
                                                                                   u64 *__restrict__ lane_stats) {
  __shared__ u32 s_vis[2 * NW * EMIT_BV];
  const u32 g = blockIdx.x % p.G, seg = blockIdx.x / p.G;
  const u32 final_mask = p.final_g ? p.final_g[g] : p.final_mask;  // per-group automata
  const u32 col = threadIdx.x >> 5, lane = lane_id();
  const u64 glane = (u64)g * (64 * NW) + col * 32 + lane;
  const u32 src = p.lanesrc[glane];
  const u32 valid_cols = __ballot_sync(FULL_MASK, src != NO_SOURCE);
  const u64 src_hi = (u64)src << 32;
  const u32 w_begin = seg * EMIT_SEG;
  const u32 n_tiles = min((u32)EMIT_TILES, (p.n - w_begin + 31) / 32);
  u64 cnt = 0, hsum = 0, hxor = 0;
  for (u32 tb = 0; tb < n_tiles; tb += EMIT_BATCH) {
    const u32 nt = min(EMIT_BATCH, n_tiles - tb);
    u64 pre[4];
    batch_fetch<NW>(p, final_mask, g, w_begin + tb * 32, nt * 32, pre);
    __syncthreads();
    batch_store<NW>(pre, s_vis);
    __syncthreads();
    for (u32 t = 0; t < nt; t++) {
      const u32 x = s_vis[col * EMIT_BV + t * 32 + lane] & valid_cols;
      if (!__any_sync(FULL_MASK, x)) continue;
      u32 m = warp_transpose32(x);
      cnt += __popc(m);
      const u32 w0 = w_begin + (tb + t) * 32;
      for (; m; m &= m - 1) digest_add(src_hi, w0 + __ffs(m) - 1, hsum, hxor);
    }
  }
  if (cnt) {
    atomicAdd(&lane_stats[3 * glane], cnt);
    atomicAdd(&lane_stats[3 * glane + 1], hsum);
    atomicXor(&lane_stats[3 * glane + 2], hxor);
  }
}

cudaError_t launch_emit_lane_stats(int nw, const EmitParams &p, unsigned long long *lane_stats, cudaStream_t st) {
  const unsigned grid = p.segs * p.G;
  if (nw == 1)
    emit_lane_stats_kernel<1><<<grid, 64, 0, st>>>(p, lane_stats);
  else
    emit_lane_stats_kernel<4><<<grid, 256, 0, st>>>(p, lane_stats);
  return cudaGetLastError();
}

// Second pass that writes interleaved (src, dst) rows straight into a
// caller's buffer (used by the entry point that allocates nothing, at most 64
// start vertices): tile by tile, the warp transpose gives each lane its
// members in vertex order; row k goes to out[2k], out[2k + 1].
template <int NW>
__global__ void emit_pairs_kernel(const EmitParams p, u32 *__restrict__ out) {
  const u32 seg = blockIdx.x, g = blockIdx.y;
  const u32 col = threadIdx.x >> 5, lane = lane_id();
  const u32 K = 64 * NW;
  const u64 glane = (u64)g * K + col * 32 + lane;
  const u32 src = p.lanesrc[glane];
  const u32 valid_cols = __ballot_sync(FULL_MASK, src != NO_SOURCE);
  const u32 *vis32 = reinterpret_cast<const u32 *>(p.vis);
  u64 pos = p.off[glane * p.segs + seg];
  const u32 w_begin = seg * EMIT_SEG;
  for (u32 t = 0; t < EMIT_TILES; t++) {
    const u32 w0 = w_begin + t * 32;
    if (w0 >= p.n) break;
    const u32 w = w0 + lane;
    u32 x = 0;
    if (w < p.n) {
      for (u32 fm = p.final_mask; fm; fm &= fm - 1) {
        u32 q = __ffs(fm) - 1;
        u64 word = (((u64)q * p.n + w) * p.G + g) * NW;
        x |= __ldcg(vis32 + word * 2 + col);
      }
    }
    const u32 mine = warp_transpose32(x & valid_cols);
    for (u32 b = mine; b; b &= b - 1) {
      out[2 * pos] = src;
      out[2 * pos + 1] = w0 + (__ffs(b) - 1);
      pos++;
    }
  }
}

cudaError_t launch_emit_pairs(const EmitParams &p, uint32_t *out, cudaStream_t st) {
  dim3 grid(p.segs, p.G);
  emit_pairs_kernel<1><<<grid, 64, 0, st>>>(p, out);
  return cudaGetLastError();
}

cudaError_t preload_static_emit_kernels() {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, emit_count_kernel<1, false>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, emit_pairs_kernel<1>);
  return e;
}

// lane_off[i] = off[i * segs] for every lane; lane_off[n_lanes] = total.
__global__ void gather_lane_off(const u64 *__restrict__ off, u32 segs, u32 n_lanes, const u64 *__restrict__ total,
                                u64 *__restrict__ lane_off) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i <= n_lanes; i += gridDim.x * blockDim.x)
    lane_off[i] = (i == n_lanes) ? *total : off[(u64)i * segs];
}

__global__ void zero_lane_counts(u32 *__restrict__ cnt, u32 segs, u32 n_lanes, const u32 *__restrict__ lane_slot) {
  const u64 total = (u64)n_lanes * segs;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (u64)gridDim.x * blockDim.x)
    if (lane_slot[i / segs] != NO_SOURCE) cnt[i] = 0;
}

cudaError_t launch_zero_lane_counts(u32 *cnt, u32 segs, u32 n_lanes, const u32 *lane_slot, cudaStream_t st) {
  const u64 total = (u64)n_lanes * segs;
  const u64 blocks = std::min<u64>((total + 255) / 256, 152ull * 16);
  zero_lane_counts<<<(unsigned)std::max<u64>(blocks, 1), 256, 0, st>>>(cnt, segs, n_lanes, lane_slot);
  return cudaGetLastError();
}

cudaError_t launch_gather_lane_off(const u64 *off, u32 segs, u32 n_lanes, const u64 *total, u64 *lane_off,
                                   cudaStream_t st) {
  gather_lane_off<<<(n_lanes + 256) / 256, 256, 0, st>>>(off, segs, n_lanes, total, lane_off);
  return cudaGetLastError();
}

// Interleaved (src, dst) rows first .. first+count-1 of one chunk.
__global__ void expand_pairs(const u32 *__restrict__ lanesrc, const u64 *__restrict__ lane_off, u32 n_lanes,
                             const u32 *__restrict__ dst, u64 first, u64 count, u32 *__restrict__ out) {
  for (u64 k = (u64)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += (u64)gridDim.x * blockDim.x) {
    u64 r = first + k;
    // owner lane: the largest i with lane_off[i] <= r
    u32 lo = 0, hi = n_lanes;  // lane_off[lo] <= r < lane_off[hi]
    while (hi - lo > 1) {
      u32 mid = (lo + hi) >> 1;
      if (lane_off[mid] <= r)
        lo = mid;
      else
        hi = mid;
    }
    out[2 * k] = lanesrc[lo];
    out[2 * k + 1] = dst[r];
  }
}

cudaError_t launch_expand_pairs(const uint32_t *lanesrc, const u64 *lane_off, uint32_t n_lanes, const uint32_t *dst,
                                u64 first, u64 count, uint32_t *out, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  u64 blocks = (count + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  expand_pairs<<<(unsigned)blocks, 256, 0, st>>>(lanesrc, lane_off, n_lanes, dst, first, count, out);
  return cudaGetLastError();
}

}  // namespace rpq
