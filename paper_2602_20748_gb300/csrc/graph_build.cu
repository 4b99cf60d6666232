// Device graph store: per-label CSR built on the GPU.
//
// The paper keeps one grid per edge label so traversal can fetch the edges of
// one label directly (Labeled Grid Format, Section 2.4).  Here each label has
// one CSR over the whole vertex-id space, for out-edges and for in-edges.
// Construction: pack every triple into a 64-bit key (label | src | dst), LSD
// radix sort, drop adjacent duplicates (identical triples count once), then
// locate the row boundaries by binary search; the in-edge CSR repeats this with
// (label | dst | src) keys.
#include <algorithm>
#include <string>

#include "device_common.cuh"
#include "rpq_internal.h"

namespace rpq {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr size_t RS_TILE = (size_t)RS_THREADS * RS_ITEMS;

__global__ void pack_keys(const uint32_t *__restrict__ a, const uint32_t *__restrict__ b,
                          const uint16_t *__restrict__ lab, size_t m, uint32_t n, uint32_t L, int bits,
                          u64 *__restrict__ keys, u32 *__restrict__ bad) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x) {
    uint32_t x = a[i], y = b[i], l = lab[i];
    if (x >= n || y >= n || l >= L) {
      atomicOr(bad, 1u);
      x = 0;
      y = 0;
      l = 0;
    }
    keys[i] = ((u64)l << (2 * bits)) | ((u64)x << bits) | (u64)y;
  }
}

__global__ void __launch_bounds__(RS_THREADS) rs_hist(const u64 *__restrict__ keys, size_t n, int shift,
                                                      u32 *__restrict__ hist, u32 nblocks) {
  __shared__ u32 cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  size_t base = (size_t)blockIdx.x * RS_TILE;
#pragma unroll 4
  for (int r = 0; r < RS_ITEMS; r++) {
    size_t i = base + (size_t)r * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255], 1u);
  }
  __syncthreads();
  hist[(size_t)threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: keys of one tile keep their order among equal digits.
__global__ void __launch_bounds__(RS_THREADS) rs_scatter(const u64 *__restrict__ in, u64 *__restrict__ out,
                                                         size_t n, int shift, const u64 *__restrict__ offs,
                                                         u32 nblocks) {
  __shared__ u64 base[256];
  __shared__ u32 wcnt[RS_THREADS / 32][256];
  const u32 d_own = threadIdx.x;  // this thread owns digit d_own
  const u32 warp = threadIdx.x >> 5;
  base[d_own] = offs[(size_t)d_own * nblocks + blockIdx.x];
  for (int w = 0; w < RS_THREADS / 32; w++) wcnt[w][d_own] = 0;
  __syncthreads();
  size_t tile = (size_t)blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ITEMS; r++) {
    size_t i = tile + (size_t)r * RS_THREADS + threadIdx.x;
    bool valid = i < n;
    u64 key = valid ? in[i] : 0;
    u32 d = valid ? (u32)((key >> shift) & 255) : 256u;
    u32 peers = __match_any_sync(FULL_MASK, d);
    u32 rank = __popc(peers & lanemask_lt());
    if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    u32 s = 0;
    for (int w = 0; w < RS_THREADS / 32; w++) {
      u32 c = wcnt[w][d_own];
      wcnt[w][d_own] = s;
      s += c;
    }
    __syncthreads();
    if (valid) out[base[d] + wcnt[warp][d] + rank] = key;
    __syncthreads();
    base[d_own] += s;
    for (int w = 0; w < RS_THREADS / 32; w++) wcnt[w][d_own] = 0;
    __syncthreads();
  }
}

__global__ void mark_unique(const u64 *__restrict__ k, size_t m, u32 *__restrict__ flag) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x)
    flag[i] = (i == 0 || k[i] != k[i - 1]) ? 1u : 0u;
}

__global__ void compact_unique(const u64 *__restrict__ k, size_t m, const u32 *__restrict__ flag,
                               const u64 *__restrict__ pos, u64 *__restrict__ out) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x)
    if (flag[i]) out[pos[i]] = k[i];
}

// Low `bits` bits of each sorted key are the column (neighbor) id.
__global__ void extract_col(const u64 *__restrict__ k, size_t m, int bits, uint32_t *__restrict__ col) {
  u64 mask = (1ull << bits) - 1;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x)
    col[i] = (uint32_t)(k[i] & mask);
}

// off[l * (n + 1) + v] = first edge whose row (key >> bits) >= l * 2^bits + v.
__global__ void row_offsets(const u64 *__restrict__ k, size_t m, int bits, uint32_t n, uint32_t L,
                            uint32_t *__restrict__ off) {
  size_t rows = (size_t)L * (n + 1);
  for (size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x; j < rows; j += (size_t)gridDim.x * blockDim.x) {
    u64 l = j / (n + 1), v = j % (n + 1);
    u64 target = (l << bits) + v;
    size_t lo = 0, hi = m;
    while (lo < hi) {
      size_t mid = (lo + hi) >> 1;
      if ((k[mid] >> bits) < target)
        lo = mid + 1;
      else
        hi = mid;
    }
    off[j] = (uint32_t)lo;
  }
}

__global__ void label_bounds(const uint32_t *__restrict__ off, uint32_t n, uint32_t L, u32 *__restrict__ out) {
  for (uint32_t l = threadIdx.x; l < L; l += blockDim.x) {
    out[2 * l] = off[(size_t)l * (n + 1)];
    out[2 * l + 1] = off[(size_t)l * (n + 1) + n];
  }
}

// Chunks of long rows: cnt[v] = number of HCHUNK-edge chunks of row v of one
// label's CSR when the row has at least HEAVY_ROW edges, else 0.
__global__ void count_chunks(const uint32_t *__restrict__ off, uint32_t n, u32 *__restrict__ cnt) {
  for (u64 v = (u64)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (u64)gridDim.x * blockDim.x) {
    uint32_t len = off[v + 1] - off[v];
    cnt[v] = len >= HEAVY_ROW ? (len + HCHUNK - 1) / HCHUNK : 0u;
  }
}

// Chunk records (vertex, first edge, end edge) at out[3 * (base + pos[v] + c)].
__global__ void write_chunks(const uint32_t *__restrict__ off, uint32_t n, const u64 *__restrict__ pos, u64 base,
                             uint32_t *__restrict__ out) {
  for (u64 v = (u64)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (u64)gridDim.x * blockDim.x) {
    uint32_t b = off[v], len = off[v + 1] - b;
    if (len < HEAVY_ROW) continue;
    uint32_t k = (len + HCHUNK - 1) / HCHUNK;
    for (uint32_t c = 0; c < k; c++) {
      u64 r = 3 * (base + pos[v] + c);
      out[r] = (uint32_t)v;
      out[r + 1] = b + c * HCHUNK;
      out[r + 2] = min(b + (c + 1) * HCHUNK, b + len);
    }
  }
}

// (label | src | dst) -> (label | dst | src)
__global__ void swap_ends(const u64 *__restrict__ k, size_t m, int bits, u64 *__restrict__ out) {
  u64 mask = (1ull << bits) - 1;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x) {
    u64 key = k[i];
    u64 l = key >> (2 * bits), x = (key >> bits) & mask, y = key & mask;
    out[i] = (l << (2 * bits)) | (y << bits) | x;
  }
}

static unsigned grid_for(size_t n, int threads) {
  size_t b = (n + threads - 1) / threads;
  if (b > 152 * 64) b = 152 * 64;
  if (b == 0) b = 1;
  return (unsigned)b;
}

#define RPQ_TRY(expr)                                                  \
  do {                                                                 \
    cudaError_t _e = (expr);                                           \
    if (_e != cudaSuccess) {                                           \
      *msg = std::string(#expr) + ": " + cudaGetErrorString(_e);       \
      rc = RPQ_ERR_CUDA;                                               \
      goto done;                                                       \
    }                                                                  \
  } while (0)

// LSD radix sort of m keys over bits [lo_bit, hi_bit) (stable, so bits
// below lo_bit keep their order); the sorted keys end up in *a (a and b are
// swapped as needed).
static cudaError_t radix_sort_range(u64 **a, u64 **b, size_t m, int lo_bit, int hi_bit, u32 *hist, u64 *offs,
                                    u64 *tmp, cudaStream_t st) {
  u32 nb = (u32)((m + RS_TILE - 1) / RS_TILE);
  for (int shift = lo_bit; shift < hi_bit; shift += 8) {
    rs_hist<<<nb, RS_THREADS, 0, st>>>(*a, m, shift, hist, nb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = exclusive_scan_u32_to_u64(hist, offs, (size_t)nb * 256, nullptr, tmp, st);
    if (e != cudaSuccess) return e;
    rs_scatter<<<nb, RS_THREADS, 0, st>>>(*a, *b, m, shift, offs, nb);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    u64 *t = *a;
    *a = *b;
    *b = t;
  }
  return cudaSuccess;
}

static cudaError_t radix_sort(u64 **a, u64 **b, size_t m, int total_bits, u32 *hist, u64 *offs, u64 *tmp,
                              cudaStream_t st) {
  return radix_sort_range(a, b, m, 0, total_bits, hist, offs, tmp, st);
}

cudaError_t sort_keys_u64(u64 **a, u64 **b, size_t m, int lo_bit, int hi_bit, cudaStream_t st) {
  if (m <= 1) return cudaSuccess;
  u32 nb = (u32)((m + RS_TILE - 1) / RS_TILE);
  size_t hist_n = (size_t)nb * 256;
  u32 *hist = nullptr;
  u64 *offs = nullptr, *tmp = nullptr;
  cudaError_t e = cudaMallocAsync(&hist, hist_n * 4, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&offs, hist_n * 8, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&tmp, scan_tmp_words(hist_n) * 8, st);
  if (e == cudaSuccess) e = radix_sort_range(a, b, m, lo_bit, hi_bit, hist, offs, tmp, st);
  if (hist) cudaFreeAsync(hist, st);
  if (offs) cudaFreeAsync(offs, st);
  if (tmp) cudaFreeAsync(tmp, st);
  return e;
}

cudaError_t unique_keys_u64(const u64 *sorted, size_t m, u64 *out, u64 *d_count, cudaStream_t st) {
  if (m == 0) return cudaMemsetAsync(d_count, 0, 8, st);
  u32 *flag = nullptr;
  u64 *pos = nullptr, *tmp = nullptr;
  cudaError_t e = cudaMallocAsync(&flag, m * 4, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&pos, m * 8, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&tmp, scan_tmp_words(m) * 8, st);
  if (e == cudaSuccess) {
    mark_unique<<<grid_for(m, 256), 256, 0, st>>>(sorted, m, flag);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = exclusive_scan_u32_to_u64(flag, pos, m, d_count, tmp, st);
  if (e == cudaSuccess) {
    compact_unique<<<grid_for(m, 256), 256, 0, st>>>(sorted, m, flag, pos, out);
    e = cudaGetLastError();
  }
  if (flag) cudaFreeAsync(flag, st);
  if (pos) cudaFreeAsync(pos, st);
  if (tmp) cudaFreeAsync(tmp, st);
  return e;
}

static int bits_for(uint64_t n) {
  int b = 1;
  while ((1ull << b) < n) b++;
  return b;
}

// Chunk records of the long rows of every label of the CSR `off`; offs gets
// the L + 1 per-label chunk offsets.
static cudaError_t build_chunks(const uint32_t *off, uint32_t n, uint32_t L, uint32_t **chunks,
                                std::vector<uint32_t> *offs, cudaStream_t st) {
  u32 *cnt = nullptr;
  u64 *pos = nullptr, *tmp = nullptr, *dtot = nullptr;
  offs->assign(L + 1, 0);
  cudaError_t e = cudaMallocAsync(&cnt, (u64)n * 4, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&pos, (u64)n * 8, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&tmp, scan_tmp_words(n) * 8, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&dtot, 8, st);
  for (int pass = 0; pass < 2 && e == cudaSuccess; pass++) {
    if (pass == 1) {
      for (uint32_t l = 0; l < L; l++) (*offs)[l + 1] += (*offs)[l];
      e = cudaMallocAsync(chunks, 3 * (u64)std::max(1u, (*offs)[L]) * 4, st);
    }
    for (uint32_t l = 0; l < L && e == cudaSuccess; l++) {
      const uint32_t *row = off + (u64)l * (n + 1);
      count_chunks<<<grid_for(n, 256), 256, 0, st>>>(row, n, cnt);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = exclusive_scan_u32_to_u64(cnt, pos, n, dtot, tmp, st);
      if (e != cudaSuccess) break;
      if (pass == 0) {
        u64 t = 0;
        e = cudaMemcpyAsync(&t, dtot, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        (*offs)[l + 1] = (uint32_t)t;
      } else {
        write_chunks<<<grid_for(n, 256), 256, 0, st>>>(row, n, pos, (*offs)[l], *chunks);
        e = cudaGetLastError();
      }
    }
  }
  if (cnt) cudaFreeAsync(cnt, st);
  if (pos) cudaFreeAsync(pos, st);
  if (tmp) cudaFreeAsync(tmp, st);
  if (dtot) cudaFreeAsync(dtot, st);
  return e;
}

int graph_key_bits(uint32_t n, uint32_t L) { return ((L > 1) ? bits_for(L) : 0) + 2 * bits_for(n); }

int build_graph(DevGraph *g, uint32_t n, uint32_t L, uint64_t m, const uint32_t *d_src, const uint32_t *d_dst,
                const uint16_t *d_lab, cudaStream_t st, std::string *msg) {
  int rc = RPQ_OK;
  const int bits = bits_for(n);
  const int lbits = (L > 1) ? bits_for(L) : 0;
  const int total_bits = lbits + 2 * bits;
  size_t mm = m ? m : 1;
  u32 nb = (u32)((mm + RS_TILE - 1) / RS_TILE);
  size_t hist_n = (size_t)nb * 256;
  size_t tmp_words = scan_tmp_words(hist_n > mm ? hist_n : mm);
  u64 *ka = nullptr, *kb = nullptr, *pos = nullptr, *offs = nullptr, *tmp = nullptr, *dtot = nullptr;
  u32 *hist = nullptr, *flag = nullptr, *bad = nullptr;
  u32 hbad = 0;
  u64 m_u = 0;
  size_t rows = (size_t)L * (n + 1);

  RPQ_TRY(cudaMallocAsync(&ka, mm * 8, st));
  RPQ_TRY(cudaMallocAsync(&kb, mm * 8, st));
  RPQ_TRY(cudaMallocAsync(&pos, mm * 8, st));
  RPQ_TRY(cudaMallocAsync(&flag, mm * 4, st));
  RPQ_TRY(cudaMallocAsync(&hist, hist_n * 4, st));
  RPQ_TRY(cudaMallocAsync(&offs, hist_n * 8, st));
  RPQ_TRY(cudaMallocAsync(&tmp, tmp_words * 8, st));
  RPQ_TRY(cudaMallocAsync(&dtot, 8, st));
  RPQ_TRY(cudaMallocAsync(&bad, 4, st));
  RPQ_TRY(cudaMemsetAsync(bad, 0, 4, st));

  if (m) {
    pack_keys<<<grid_for(m, 256), 256, 0, st>>>(d_src, d_dst, d_lab, m, n, L, bits, ka, bad);
    RPQ_TRY(cudaGetLastError());
    RPQ_TRY(cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, st));
    RPQ_TRY(cudaStreamSynchronize(st));
    if (hbad) {
      *msg = "edge endpoint or label out of range";
      rc = RPQ_ERR_INVALID_ARG;
      goto done;
    }
    RPQ_TRY(radix_sort(&ka, &kb, m, total_bits, hist, offs, tmp, st));
    mark_unique<<<grid_for(m, 256), 256, 0, st>>>(ka, m, flag);
    RPQ_TRY(cudaGetLastError());
    RPQ_TRY(exclusive_scan_u32_to_u64(flag, pos, m, dtot, tmp, st));
    compact_unique<<<grid_for(m, 256), 256, 0, st>>>(ka, m, flag, pos, kb);
    RPQ_TRY(cudaGetLastError());
    RPQ_TRY(cudaMemcpyAsync(&m_u, dtot, 8, cudaMemcpyDeviceToHost, st));
    RPQ_TRY(cudaStreamSynchronize(st));
    {
      u64 *t = ka;
      ka = kb;
      kb = t;
    }
  }
  g->n = n;
  g->L = L;
  g->m = m_u;
  RPQ_TRY(cudaMallocAsync(&g->out_off, rows * 4, st));
  RPQ_TRY(cudaMallocAsync(&g->in_off, rows * 4, st));
  RPQ_TRY(cudaMallocAsync(&g->out_col, (m_u ? m_u : 1) * 4, st));
  RPQ_TRY(cudaMallocAsync(&g->in_col, (m_u ? m_u : 1) * 4, st));
  // out-edges: ka holds distinct (label | src | dst) keys in order
  extract_col<<<grid_for(m_u ? m_u : 1, 256), 256, 0, st>>>(ka, m_u, bits, g->out_col);
  RPQ_TRY(cudaGetLastError());
  row_offsets<<<grid_for(rows, 256), 256, 0, st>>>(ka, m_u, bits, n, L, g->out_off);
  RPQ_TRY(cudaGetLastError());
  // in-edges
  if (m_u) {
    swap_ends<<<grid_for(m_u, 256), 256, 0, st>>>(ka, m_u, bits, kb);
    RPQ_TRY(cudaGetLastError());
    {
      u64 *t = ka;
      ka = kb;
      kb = t;
    }
    RPQ_TRY(radix_sort(&ka, &kb, m_u, total_bits, hist, offs, tmp, st));
  }
  extract_col<<<grid_for(m_u ? m_u : 1, 256), 256, 0, st>>>(ka, m_u, bits, g->in_col);
  RPQ_TRY(cudaGetLastError());
  row_offsets<<<grid_for(rows, 256), 256, 0, st>>>(ka, m_u, bits, n, L, g->in_off);
  RPQ_TRY(cudaGetLastError());
  {
    // per-label edge counts: off[l * (n + 1) + n] - off[l * (n + 1)]
    label_bounds<<<1, 64, 0, st>>>(g->out_off, n, L, hist);
    RPQ_TRY(cudaGetLastError());
    std::vector<uint32_t> ends(2 * L);
    RPQ_TRY(cudaMemcpyAsync(ends.data(), hist, 8 * L, cudaMemcpyDeviceToHost, st));
    RPQ_TRY(cudaStreamSynchronize(st));
    g->label_edges.assign(L, 0);
    for (uint32_t l = 0; l < L; l++) g->label_edges[l] = (uint64_t)ends[2 * l + 1] - ends[2 * l];
  }
  RPQ_TRY(build_chunks(g->in_off, n, L, &g->hchunk_in, &g->hchunk_in_off, st));
  RPQ_TRY(build_chunks(g->out_off, n, L, &g->hchunk_out, &g->hchunk_out_off, st));
done:
  if (ka) cudaFreeAsync(ka, st);
  if (kb) cudaFreeAsync(kb, st);
  if (pos) cudaFreeAsync(pos, st);
  if (flag) cudaFreeAsync(flag, st);
  if (hist) cudaFreeAsync(hist, st);
  if (offs) cudaFreeAsync(offs, st);
  if (tmp) cudaFreeAsync(tmp, st);
  if (dtot) cudaFreeAsync(dtot, st);
  if (bad) cudaFreeAsync(bad, st);
  return rc;
}

}  // namespace rpq
