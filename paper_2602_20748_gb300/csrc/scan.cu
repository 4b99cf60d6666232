// Device-wide exclusive prefix sums (tile reduce -> recursive scan of tile
// sums -> tile apply).  Used for list compaction, radix-sort offsets and
// result offsets.
#include "device_common.cuh"
#include "rpq_internal.h"

namespace rpq {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr size_t SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename TIn>
__global__ void __launch_bounds__(SCAN_THREADS) scan_tile_sums(const TIn *__restrict__ in, size_t n,
                                                                u64 *__restrict__ sums) {
  size_t base = (size_t)blockIdx.x * SCAN_TILE;
  u64 s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++) {
    size_t i = base + (size_t)k * SCAN_THREADS + threadIdx.x;
    if (i < n) s += (u64)in[i];
  }
  s = warp_sum(s);
  __shared__ u64 ws[SCAN_THREADS / 32];
  if (lane_id() == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    u64 t = 0;
    for (int w = 0; w < SCAN_THREADS / 32; w++) t += ws[w];
    sums[blockIdx.x] = t;
  }
}

// Exclusive scan of one tile, plus the tile's offset.  Block 0 of a
// single-tile scan also writes the total.
template <typename TIn>
__global__ void __launch_bounds__(SCAN_THREADS) scan_tile_apply(const TIn *__restrict__ in, u64 *__restrict__ out,
                                                                 size_t n, const u64 *__restrict__ tile_off,
                                                                 u64 *__restrict__ total) {
  __shared__ u64 buf[SCAN_TILE];
  __shared__ u64 ws[SCAN_THREADS / 32];
  size_t base = (size_t)blockIdx.x * SCAN_TILE;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++) {
    size_t i = base + (size_t)k * SCAN_THREADS + threadIdx.x;
    buf[k * SCAN_THREADS + threadIdx.x] = (i < n) ? (u64)in[i] : 0;
  }
  __syncthreads();
  u64 v[SCAN_ITEMS];
  u64 local = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++) {
    v[k] = buf[threadIdx.x * SCAN_ITEMS + k];
    local += v[k];
  }
  // inclusive warp scan of per-thread sums
  u64 inc = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    u64 t = __shfl_up_sync(FULL_MASK, inc, o);
    if (lane_id() >= (u32)o) inc += t;
  }
  if (lane_id() == 31) ws[threadIdx.x >> 5] = inc;
  __syncthreads();
  u64 warp_off = 0, block_total = 0;
  for (int w = 0; w < SCAN_THREADS / 32; w++) {
    u64 t = ws[w];
    if (w < (int)(threadIdx.x >> 5)) warp_off += t;
    block_total += t;
  }
  u64 run = (tile_off ? tile_off[blockIdx.x] : 0) + warp_off + inc - local;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++) {
    buf[threadIdx.x * SCAN_ITEMS + k] = run;
    run += v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; k++) {
    size_t i = base + (size_t)k * SCAN_THREADS + threadIdx.x;
    if (i < n) out[i] = buf[k * SCAN_THREADS + threadIdx.x];
  }
  if (total && tile_off == nullptr && blockIdx.x == 0 && threadIdx.x == 0) *total = block_total;
}

size_t scan_tmp_words(size_t n) {
  size_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (nb <= 1) return 1;
  return nb + scan_tmp_words(nb);
}

template <typename TIn>
static cudaError_t scan_impl(const TIn *in, u64 *out, size_t n, u64 *total, u64 *tmp, cudaStream_t st) {
  if (n == 0) {
    if (total) return cudaMemsetAsync(total, 0, sizeof(u64), st);
    return cudaSuccess;
  }
  size_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (nb == 1) {
    scan_tile_apply<TIn><<<1, SCAN_THREADS, 0, st>>>(in, out, n, nullptr, total);
    return cudaGetLastError();
  }
  u64 *sums = tmp;
  scan_tile_sums<TIn><<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, n, sums);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = scan_impl<u64>(sums, sums, nb, total, tmp + nb, st);
  if (e != cudaSuccess) return e;
  scan_tile_apply<TIn><<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, out, n, sums, nullptr);
  return cudaGetLastError();
}

cudaError_t exclusive_scan_u32_to_u64(const uint32_t *in, u64 *out, size_t n, u64 *total, u64 *tmp,
                                      cudaStream_t st) {
  return scan_impl<uint32_t>(in, out, n, total, tmp, st);
}

cudaError_t exclusive_scan_u64(const u64 *in, u64 *out, size_t n, u64 *total, u64 *tmp, cudaStream_t st) {
  return scan_impl<u64>(in, out, n, total, tmp, st);
}

cudaError_t preload_scan_kernels() {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, scan_tile_sums<uint32_t>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, scan_tile_apply<uint32_t>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, scan_tile_sums<u64>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, scan_tile_apply<u64>);
  return e;
}

}  // namespace rpq
