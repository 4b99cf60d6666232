// Small device helpers shared by the RPQ kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rpq {

typedef unsigned long long u64;
typedef unsigned int u32;

constexpr u32 FULL_MASK = 0xffffffffu;
constexpr u32 NO_SOURCE = 0xffffffffu;

__device__ __forceinline__ u32 lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ u32 lanemask_lt() {
  u32 m;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ u64 globaltimer_ns() {
  u64 t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// SplitMix64 output for state x (Steele, Lea and Flood, OOPSLA 2014): add the
// golden-ratio increment, then the variant-13 64-bit finalizer.
__host__ __device__ __forceinline__ u64 splitmix64(u64 x) {
  u64 z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
  return v;
}

__device__ __forceinline__ u64 warp_xor(u64 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v ^= __shfl_xor_sync(FULL_MASK, v, o);
  return v;
}

}  // namespace rpq
