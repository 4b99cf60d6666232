// run_rpq_static: an RPQ entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc (or any allocator) when they run a
// query: a host application that hands the whole device memory to its own
// pool or buffer manager up front, a latency-critical loop that must not take
// the device-wide synchronization an allocation can imply, or a plug-in that
// runs inside another runtime which forbids allocating on its device.  For
// them this file keeps the traversal's scratch memory in one file-scope
// device array and runs the same traversal and emission kernels as run_rpq
// (one lane group of up to 64 start vertices) on it.  The caller passes the
// inputs (a loaded graph, a compiled query, start vertices) and the output
// buffer.
//
// The array belongs to this file's device module.  Under the runtime's lazy
// module loading that module, and with it the array, is loaded the first time
// the host asks for the array's address; rpq_create does that (with the
// context's device current) and also loads the kernels this entry point
// launches, so the array is reserved when the first context on a device is
// created and a later call has nothing left to reserve.
//
// Every call shares the one array, so calls whose GPU work overlaps (other
// threads, other streams of the same device) race with each other; callers
// serialize them.  The array keeps the previous call's contents; everything a
// call needs zeroed is cleared by the call itself.
#include <cstring>

#include "crpq.h"
#include "device_common.cuh"
#include "rpq_internal.h"

namespace rpq {
namespace {

constexpr size_t STATIC_SCRATCH_BYTES = 64ull << 20;  // 64 MiB per device

static __device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

// Bytes of g_static_scratch a query with Q states on n vertices needs.
static size_t static_scratch_need(uint32_t Q, uint32_t n, uint32_t segs) {
  size_t words = (size_t)Q * n;
  size_t need = 0;
  need += align256(sizeof(BfsCtl));
  need += align256(4 * sizeof(u64));    // digest sum, xor, total, spare
  need += align256(64 * sizeof(u32));   // lanesrc
  need += align256(sizeof(u64));        // empty-lane mask
  need += 5 * align256(words * 8);      // VIS, two frontiers, two entry lists
  need += align256((size_t)64 * segs * 4);  // per (lane, segment) counts
  need += align256((size_t)64 * segs * 8);  // their offsets
  need += align256(scan_tmp_words((size_t)64 * segs) * 8);
  return need;
}

// Set-up for one context, with its device current: the host-side name of the
// array is not a device address, so the runtime is asked for the address
// (which also loads the array's module); the kernels run_rpq_static launches
// are loaded too.  Each context keeps its own copy of the address, so no
// state is shared between threads, and a context created after a
// cudaDeviceReset looks the address up afresh.
int static_scratch_prepare(void **addr, std::string *msg) {
  *addr = nullptr;
  void *a = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&a, g_static_scratch);
  if (e != cudaSuccess || !a) {
    *msg = std::string("cudaGetSymbolAddress of the static scratch: ") + cudaGetErrorString(e);
    return RPQ_ERR_CUDA;
  }
  if ((e = preload_static_msbfs_kernels()) != cudaSuccess || (e = preload_static_emit_kernels()) != cudaSuccess ||
      (e = preload_scan_kernels()) != cudaSuccess) {
    *msg = std::string("loading the kernels of run_rpq_static: ") + cudaGetErrorString(e);
    return RPQ_ERR_CUDA;
  }
  *addr = a;
  return RPQ_OK;
}

}  // namespace rpq

using namespace rpq;

extern "C" int run_rpq_static(rpq_ctx *ctx, const rpq_graph *g, const rpq_query *q, const uint32_t *sources,
                              uint32_t n_sources, uint32_t *out_pairs, uint64_t max_rows, uint64_t *n_rows) {
  if (!ctx || !g || !q || !sources || !n_rows || (!out_pairs && max_rows))
    return ctx ? ctx_error(ctx, RPQ_ERR_INVALID_ARG, "null argument") : RPQ_ERR_INVALID_ARG;
  *n_rows = 0;
  const int dev = ctx_device(ctx);
  if (dev < 0) return ctx_error(ctx, RPQ_ERR_NO_DEVICE, "host-only context has no GPU");
  if (n_sources == 0 || n_sources > 64)
    return ctx_error(ctx, RPQ_ERR_INVALID_ARG, "run_rpq_static takes 1 to 64 start vertices");
  const DevGraph &dg = graph_dev(g);
  const QueryDesc &qd = query_host(q).d;

  // sorted distinct start vertices, on the stack
  uint32_t src[64];
  uint32_t ns = 0;
  for (uint32_t i = 0; i < n_sources; i++) {
    uint32_t s = sources[i];
    if (s >= dg.n) return ctx_error(ctx, RPQ_ERR_INVALID_ARG, "source id out of range");
    uint32_t j = ns;
    while (j > 0 && src[j - 1] > s) j--;
    if (j > 0 && src[j - 1] == s) continue;
    for (uint32_t k = ns; k > j; k--) src[k] = src[k - 1];
    src[j] = s;
    ns++;
  }
  const uint32_t Q = qd.n_states;
  if (Q == 0) return RPQ_OK;  // empty language: no rows
  const uint32_t n = dg.n;
  const uint32_t segs = (n + EMIT_SEG - 1) / EMIT_SEG;
  const size_t need = static_scratch_need(Q, n, segs);
  if (need > STATIC_SCRATCH_BYTES)
    return ctx_error(ctx, RPQ_ERR_OUT_OF_BUDGET,
                     "run_rpq_static: this graph and query need " + std::to_string(need) +
                         " bytes of scratch; the static scratch holds " + std::to_string(STATIC_SCRATCH_BYTES) +
                         " (about 40 * states * vertices bytes are needed)");

  cudaError_t e = cudaSetDevice(dev);
  if (e != cudaSuccess) return ctx_error(ctx, RPQ_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  // the array's device address, found when the context was created
  unsigned char *base = static_cast<unsigned char *>(ctx_static_scratch(ctx));
  if (!base) return ctx_error(ctx, RPQ_ERR_CUDA, "the context has no static scratch address");
  size_t at = 0;
  auto take = [&](size_t bytes) {
    unsigned char *p = base + at;
    at += align256(bytes);
    return p;
  };
  const size_t words = (size_t)Q * n;
  BfsCtl *ctl = (BfsCtl *)take(sizeof(BfsCtl));
  u64 *small = (u64 *)take(4 * sizeof(u64));
  u32 *lanesrc = (u32 *)take(64 * sizeof(u32));
  u64 *empty = (u64 *)take(sizeof(u64));
  u64 *vis = (u64 *)take(words * 8);
  u64 *fr0 = (u64 *)take(words * 8);
  u64 *fr1 = (u64 *)take(words * 8);
  u64 *list0 = (u64 *)take(words * 8);
  u64 *list1 = (u64 *)take(words * 8);
  u32 *cnt = (u32 *)take((size_t)64 * segs * 4);
  u64 *off = (u64 *)take((size_t)64 * segs * 8);
  u64 *tmp = (u64 *)take(scan_tmp_words((size_t)64 * segs) * 8);

  cudaStream_t st = ctx_stream(ctx);
  uint32_t lanes[64];
  uint64_t empty_mask = 0;
  for (uint32_t i = 0; i < 64; i++) {
    lanes[i] = i < ns ? src[i] : NO_SOURCE;
    if (i >= ns) empty_mask |= 1ull << i;
  }
#define STATIC_CK(expr)                                                                                 \
  do {                                                                                                  \
    cudaError_t _e = (expr);                                                                            \
    if (_e != cudaSuccess) return ctx_error(ctx, RPQ_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
  } while (0)
  // what must start at zero: control block, digest / total, both frontiers
  STATIC_CK(cudaMemsetAsync(ctl, 0, sizeof(BfsCtl), st));
  STATIC_CK(cudaMemsetAsync(small, 0, 4 * sizeof(u64), st));
  STATIC_CK(cudaMemsetAsync(fr0, 0, words * 8, st));
  STATIC_CK(cudaMemsetAsync(fr1, 0, words * 8, st));
  STATIC_CK(cudaMemcpyAsync(lanesrc, lanes, sizeof(lanes), cudaMemcpyHostToDevice, st));
  STATIC_CK(cudaMemcpyAsync(empty, &empty_mask, sizeof(empty_mask), cudaMemcpyHostToDevice, st));

  BfsParams p;
  std::memset(&p, 0, sizeof(p));
  p.out_off = dg.out_off;
  p.out_col = dg.out_col;
  p.in_off = dg.in_off;
  p.in_col = dg.in_col;
  p.n = n;
  p.L = dg.L;
  p.G = 1;
  p.Q = Q;
  p.lanesrc = lanesrc;
  p.vis = vis;
  p.fr0 = fr0;
  p.fr1 = fr1;
  p.claim = nullptr;  // one 64-bit word per lane group: claims come from the OR itself
  p.list0 = list0;
  p.list1 = list1;
  p.list_cap = words;  // one append per (state, vertex) per level (no segments here)
  p.append_seg = 0;
  p.ctl = ctl;
  p.stamp_base = 0;
  const int blocks = ctx_bfs_blocks(ctx, 1);
  if (blocks <= 0) return ctx_error(ctx, RPQ_ERR_CUDA, "traversal kernel cannot be made resident");
  p.nblocks = (unsigned)blocks;
  p.force = 0;
  p.alpha = ctx_alpha(ctx);
  p.pull_dynamic = 1;
  p.lane_by_source = 1;
  p.hchunk = nullptr;  // long rows are scanned in place
  for (uint32_t l = 0; l < dg.L; l++) p.label_edges[l] = dg.label_edges[l];
  p.time_limit_ns = ctx_time_limit_ns(ctx);
  p.q = qd;
  STATIC_CK(launch_vis_init(1, p, empty, st));
  STATIC_CK(launch_msbfs(1, p, blocks, 256, st));

  EmitParams ep{};
  ep.vis = vis;
  ep.n = n;
  ep.G = 1;
  ep.Q = Q;
  ep.final_mask = qd.final_mask;
  ep.lanesrc = lanesrc;
  ep.segs = segs;
  ep.cnt = cnt;
  ep.off = off;
  ep.dst = nullptr;
  ep.digest = small;
  STATIC_CK(launch_emit(1, false, false, ep, st));
  STATIC_CK(exclusive_scan_u32_to_u64(cnt, off, (size_t)64 * segs, small + 2, tmp, st));
  unsigned int err = 0;
  u64 total = 0;
  STATIC_CK(cudaMemcpyAsync(&err, &ctl->err, sizeof(err), cudaMemcpyDeviceToHost, st));
  STATIC_CK(cudaMemcpyAsync(&total, small + 2, sizeof(total), cudaMemcpyDeviceToHost, st));
  STATIC_CK(cudaStreamSynchronize(st));
  if (err == ERR_LIST_OVERFLOW) return ctx_error(ctx, RPQ_ERR_CUDA, "internal: traversal entry list overflow");
  if (err) return ctx_error(ctx, RPQ_ERR_TIMEOUT, "traversal grid barrier wait ran out of time");
  *n_rows = total;
  if (total > max_rows)
    return ctx_error(ctx, RPQ_ERR_OUT_OF_BUDGET,
                     "run_rpq_static: the result has " + std::to_string(total) + " rows, the output buffer holds " +
                         std::to_string(max_rows));
  if (total) {
    STATIC_CK(launch_emit_pairs(ep, out_pairs, st));
    STATIC_CK(cudaStreamSynchronize(st));
  }
#undef STATIC_CK
  return RPQ_OK;
}
