// Edge lists for the start-in-the-middle plan (Section 2.3 WavePlan, plan
// A3; executed as A5, Section 6.3): the pairs of a materialized sub-RPQ
// R(beta) become the edges of one extra label of a temporary graph, next to
// the graph's own edges, so that alpha . beta can then be evaluated as
// alpha . X by the ordinary traversal.  These kernels write (src, dst,
// label) triples that the graph builder sorts into per-label CSR.
#include "device_common.cuh"
#include "rpq_internal.h"

namespace rpq {

// One thread per (label, vertex) row of the out-CSR: its edges as triples at
// their CSR positions (out_col index e is triple e).
__global__ void csr_triples_kernel(const u32 *__restrict__ off, const u32 *__restrict__ col, u32 n, u32 L,
                                   u32 *__restrict__ src, u32 *__restrict__ dst, unsigned short *__restrict__ lab) {
  const u64 rows = (u64)L * n;
  for (u64 r = (u64)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (u64)gridDim.x * blockDim.x) {
    const u32 l = (u32)(r / n), v = (u32)(r % n);
    const u32 *o = off + (u64)l * (n + 1) + v;
    for (u32 e = o[0]; e < o[1]; e++) {
      src[e] = v;
      dst[e] = col[e];
      lab[e] = (unsigned short)l;
    }
  }
}

// One warp per lane of a materialized chunk: the lane's rows (s, y) as
// triples (s, y, x) from position base + lane_off[lane].
__global__ void chunk_triples_kernel(const u32 *__restrict__ lanesrc, const u64 *__restrict__ lane_off, u32 n_lanes,
                                     const u32 *__restrict__ cdst, u64 base, unsigned short x,
                                     u32 *__restrict__ src, u32 *__restrict__ dst, unsigned short *__restrict__ lab) {
  const u64 warp = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
  for (u64 i = warp; i < n_lanes; i += nwarps) {
    const u32 s = lanesrc[i];
    const u64 b = lane_off[i], e = lane_off[i + 1];
    if (s == NO_SOURCE) continue;
    for (u64 k = b + lane_id(); k < e; k += 32) {
      src[base + k] = s;
      dst[base + k] = cdst[k];
      lab[base + k] = x;
    }
  }
}

cudaError_t launch_csr_triples(const uint32_t *off, const uint32_t *col, uint32_t n, uint32_t L, uint32_t *src,
                               uint32_t *dst, uint16_t *lab, cudaStream_t st) {
  const u64 rows = (u64)L * n;
  if (rows == 0) return cudaSuccess;
  u64 blocks = (rows + 255) / 256;
  if (blocks > 152ull * 64) blocks = 152ull * 64;
  csr_triples_kernel<<<(unsigned)blocks, 256, 0, st>>>(off, col, n, L, src, dst,
                                                        reinterpret_cast<unsigned short *>(lab));
  return cudaGetLastError();
}

cudaError_t launch_chunk_triples(const uint32_t *lanesrc, const unsigned long long *lane_off, uint32_t n_lanes,
                                 const uint32_t *cdst, unsigned long long base, uint16_t x, uint32_t *src,
                                 uint32_t *dst, uint16_t *lab, cudaStream_t st) {
  if (n_lanes == 0) return cudaSuccess;
  u64 blocks = ((u64)n_lanes * 32 + 255) / 256;
  if (blocks > 152ull * 32) blocks = 152ull * 32;
  chunk_triples_kernel<<<(unsigned)blocks, 256, 0, st>>>(lanesrc, lane_off, n_lanes, cdst, base,
                                                          (unsigned short)x, src, dst,
                                                          reinterpret_cast<unsigned short *>(lab));
  return cudaGetLastError();
}

}  // namespace rpq
