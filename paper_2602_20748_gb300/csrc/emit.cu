// Result emission: visited words -> distinct (src, dst) rows in sorted order.
//
// After the search, the result set of start vertex s (Definition 1) is the
// set of v with some accepting state q such that s's lane is set in the
// visited word of (group g, state q, vertex v).  For lane group g, OR the
// accepting states' words into a K-bit result word per vertex.  A block owns
// a segment of EMIT_SEG vertices of one group; warp c handles lane column c
// (32 lanes) and walks the segment in 32-vertex tiles, thread i holding the
// 32 lane bits of vertex w0 + i.  For every lane j with a bit in the tile, a
// ballot over bit j gives the tile's members of lane j's row in vertex order:
// the count pass adds its popcount to lane j's (lane, segment) count, and the
// write pass stores the members at consecutive positions of lane j's row (one
// coalesced store per lane and tile).  An exclusive scan over the counts laid
// out [lane][segment] gives every row its output position directly (lanes
// are in source order, segments in vertex order).  The row digest is folded
// by the thread that holds the member.
#include "device_common.cuh"
#include "rpq_internal.h"

namespace rpq {

template <int NW, bool WRITE, bool DIGEST>
__global__ void emit_kernel(const EmitParams p) {
  // groups of one segment are adjacent blocks, so they read the same
  // visited lines close together in time
  const u32 g = blockIdx.x % p.G, seg = blockIdx.x / p.G;
  const u32 col = threadIdx.x >> 5, lane = lane_id();
  const u32 K = 64 * NW;
  const u64 glane = (u64)g * K + col * 32 + lane;
  const u32 src = p.lanesrc[glane];
  const u32 valid_cols = __ballot_sync(FULL_MASK, src != NO_SOURCE);
  const u32 *vis32 = reinterpret_cast<const u32 *>(p.vis);
  const u32 lt = (1u << lane) - 1u;
  u64 cnt = 0, hsum = 0, hxor = 0;
  // count pass: per-lane counts of this thread's vertices as bit planes
  // (EMIT_TILES <= 2^CNT_PLANES - 1 vertices per thread)
  constexpr int CNT_PLANES = 8;
  static_assert(EMIT_TILES < (1 << CNT_PLANES), "count planes too narrow");
  u32 planes[CNT_PLANES];
#pragma unroll
  for (int k = 0; k < CNT_PLANES; k++) planes[k] = 0;
  u64 pos = 0;  // lane `lane`'s next output position (write pass)
  if (WRITE) pos = p.off[glane * p.segs + seg];
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
    x &= valid_cols;
    if (!WRITE && !DIGEST) {
      // count only: add x into per-thread bit-sliced counters (plane k holds
      // bit k of each lane's count over this thread's vertices so far)
      u32 carry = x;
#pragma unroll
      for (int k = 0; k < CNT_PLANES; k++) {
        const u32 t = planes[k] & carry;
        planes[k] ^= carry;
        carry = t;
      }
      continue;
    }
    for (u32 rows = __reduce_or_sync(FULL_MASK, x); rows; rows &= rows - 1) {
      const u32 j = __ffs(rows) - 1;
      const u32 mine = (x >> j) & 1u;
      const u32 m = __ballot_sync(FULL_MASK, mine);
      if (WRITE) {
        const u64 base = __shfl_sync(FULL_MASK, pos, j);
        if (mine) p.dst[base + __popc(m & lt)] = w;
      }
      if (DIGEST) {
        const u32 sj = __shfl_sync(FULL_MASK, src, j);
        if (mine) {
          u64 h = splitmix64(((u64)sj << 32) | (u64)w);
          hsum += h;
          hxor ^= h;
        }
      }
      if (lane == j) {
        if (WRITE)
          pos += __popc(m);
        else
          cnt += __popc(m);
      }
    }
  }
  if (!WRITE && !DIGEST) {
    // lane j's count = sum over planes k of 2^k * (threads with bit j set in
    // plane k): transpose each plane with 32 ballots
#pragma unroll
    for (int k = 0; k < CNT_PLANES; k++) {
      if (!__any_sync(FULL_MASK, planes[k])) continue;
      u32 mine = 0;
#pragma unroll
      for (int j = 0; j < 32; j++) {
        const u32 b = __ballot_sync(FULL_MASK, (planes[k] >> j) & 1u);
        if (lane == (u32)j) mine = b;
      }
      cnt += (u64)__popc(mine) << k;
    }
  }
  if (!WRITE) p.cnt[glane * p.segs + seg] = (u32)cnt;
  if (DIGEST) {
    hsum = warp_sum(hsum);
    hxor = warp_xor(hxor);
    if (lane == 0 && (hsum | hxor)) {
      atomicAdd(&p.digest[0], hsum);
      atomicXor(&p.digest[1], hxor);
    }
  }
}

// Pass 1 (write = false) counts per (lane, segment); pass 2 (write = true)
// writes the destinations.  The row digest is folded in the pass given
// digest = true (the write pass when rows are kept, else the count pass).
cudaError_t launch_emit(int nw, bool write, bool digest, const EmitParams &p, cudaStream_t st) {
  const unsigned grid = p.segs * p.G;
  const int threads = nw == 1 ? 64 : 256;
  if (nw == 1) {
    if (write)
      digest ? emit_kernel<1, true, true><<<grid, threads, 0, st>>>(p)
             : emit_kernel<1, true, false><<<grid, threads, 0, st>>>(p);
    else
      digest ? emit_kernel<1, false, true><<<grid, threads, 0, st>>>(p)
             : emit_kernel<1, false, false><<<grid, threads, 0, st>>>(p);
  } else {
    if (write)
      digest ? emit_kernel<4, true, true><<<grid, threads, 0, st>>>(p)
             : emit_kernel<4, true, false><<<grid, threads, 0, st>>>(p);
    else
      digest ? emit_kernel<4, false, true><<<grid, threads, 0, st>>>(p)
             : emit_kernel<4, false, false><<<grid, threads, 0, st>>>(p);
  }
  return cudaGetLastError();
}

// Digest of a materialized chunk's rows: block b takes lanes b, b +
// gridDim.x, ...; the rows of lane i are contiguous (dst[lane_off[i] ..
// lane_off[i + 1])) and all belong to source lanesrc[i].  The 16-byte aligned
// middle of a lane's rows is read four rows per load, two loads in flight per
// thread; the unaligned ends row by row.
__device__ __forceinline__ void digest_add(u64 src, u32 y, u64 &hsum, u64 &hxor) {
  const u64 h = splitmix64(src | (u64)y);
  hsum += h;
  hxor ^= h;
}

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
__global__ void emit_lane_stats_kernel(const EmitParams p, u64 *__restrict__ lane_stats) {
  const u32 g = blockIdx.x % p.G, seg = blockIdx.x / p.G;
  const u32 final_mask = p.final_g ? p.final_g[g] : p.final_mask;  // per-group automata
  const u32 col = threadIdx.x >> 5, lane = lane_id();
  const u32 K = 64 * NW;
  const u64 glane = (u64)g * K + col * 32 + lane;
  const u32 src = p.lanesrc[glane];
  const u32 valid_cols = __ballot_sync(FULL_MASK, src != NO_SOURCE);
  const u32 *vis32 = reinterpret_cast<const u32 *>(p.vis);
  u64 cnt = 0, hsum = 0, hxor = 0;
  const u32 w_begin = seg * EMIT_SEG;
  for (u32 t = 0; t < EMIT_TILES; t++) {
    const u32 w0 = w_begin + t * 32;
    if (w0 >= p.n) break;
    const u32 w = w0 + lane;
    u32 x = 0;
    if (w < p.n) {
      for (u32 fm = final_mask; fm; fm &= fm - 1) {
        u32 q = __ffs(fm) - 1;
        u64 word = (((u64)q * p.n + w) * p.G + g) * NW;
        x |= __ldcg(vis32 + word * 2 + col);
      }
    }
    x &= valid_cols;
    if (!__any_sync(FULL_MASK, x)) continue;
    u32 mine = 0;
#pragma unroll
    for (int j = 0; j < 32; j++) {
      u32 b = __ballot_sync(FULL_MASK, (x >> j) & 1u);
      if (lane == (u32)j) mine = b;
    }
    cnt += __popc(mine);
    for (u32 b = mine; b; b &= b - 1) {
      u64 h = splitmix64(((u64)src << 32) | (u64)(w0 + __ffs(b) - 1));
      hsum += h;
      hxor ^= h;
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
// caller's buffer (used by the entry point that allocates nothing): same walk
// as emit_kernel's write pass, row k at out[2k], out[2k + 1].
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
    x &= valid_cols;
    u32 mine = 0;
#pragma unroll
    for (int j = 0; j < 32; j++) {
      u32 b = __ballot_sync(FULL_MASK, (x >> j) & 1u);
      if (lane == (u32)j) mine = b;
    }
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

// lane_off[i] = off[i * segs] for every lane; lane_off[n_lanes] = total.
__global__ void gather_lane_off(const u64 *__restrict__ off, u32 segs, u32 n_lanes, const u64 *__restrict__ total,
                                u64 *__restrict__ lane_off) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i <= n_lanes; i += gridDim.x * blockDim.x)
    lane_off[i] = (i == n_lanes) ? *total : off[(u64)i * segs];
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
