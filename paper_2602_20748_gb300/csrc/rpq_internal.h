// Internal declarations shared by the host API and the CUDA kernels of the
// RPQ engine.  Not part of the public ABI (see include/rpq.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rpq.h"

namespace rpq {

// ---------------------------------------------------------------------------
// Compiled query: the minimal DFA in the forms the kernels use.
// ---------------------------------------------------------------------------
struct QueryDesc {
  uint32_t n_states;    // 0 means the empty language
  uint32_t final_mask;  // bit q: state q accepts
  uint32_t n_labels;    // largest label id used + 1
  uint32_t n_trans;
  // Top-down form: transitions leaving state q are [out_begin[q], out_begin[q+1]).
  uint16_t out_begin[RPQ_MAX_STATES + 1];
  uint8_t out_label[RPQ_MAX_TRANSITIONS];
  uint8_t out_to[RPQ_MAX_TRANSITIONS];
  // Bottom-up form: for target state q, groups [in_begin[q], in_begin[q+1]) of
  // (label, bitmask of source states that reach q on that label).
  uint16_t in_begin[RPQ_MAX_STATES + 1];
  uint8_t in_label[RPQ_MAX_TRANSITIONS];
  uint32_t in_from[RPQ_MAX_TRANSITIONS];
};

// Host-side compiled query.
struct HostQuery {
  QueryDesc d;
  std::vector<int32_t> next;  // n_states * n_labels, -1 = none
  // Minimal DFA of the reversed language, for evaluation from the target end
  // over in-edges (absent when it would exceed RPQ_MAX_STATES).
  bool has_rev = false;
  QueryDesc rev;
  std::vector<int32_t> rev_next;
};

// Parses and compiles; returns RPQ_OK or an error code with *msg set.
int compile_regex(const char *regex, const char *const *names, uint32_t n_names, HostQuery *out, std::string *msg);
// The minimal DFA of L(alpha) followed by one edge of label x (x above every
// label alpha uses).
int dfa_then_label(const HostQuery &alpha, uint32_t x, HostQuery *out, std::string *msg);

// ---------------------------------------------------------------------------
// Device-resident graph: one CSR per edge label over the full id space, for
// out-edges (sorted by label, src, dst) and in-edges (label, dst, src).
// off[l * (n + 1) + v] is the first edge of row v of label l.
// ---------------------------------------------------------------------------
// In-edge rows with at least HEAVY_ROW edges are cut into chunks of HCHUNK
// edges at graph load; bottom-up levels share the chunks among all warps
// instead of scanning such a row with one warp.
constexpr uint32_t HEAVY_ROW = 128;
constexpr uint32_t HCHUNK = 256;

struct DevGraph {
  uint32_t n = 0;
  uint32_t L = 0;
  uint64_t m = 0;
  uint32_t *out_off = nullptr;
  uint32_t *out_col = nullptr;
  uint32_t *in_off = nullptr;
  uint32_t *in_col = nullptr;
  uint8_t *vlabel = nullptr;
  // Chunks (vertex, first edge, end edge) of the rows with >= HEAVY_ROW
  // edges, per direction, grouped by label: label l's chunks are
  // [off[l], off[l+1]) (host copy of the L+1 offsets).
  uint32_t *hchunk_in = nullptr, *hchunk_out = nullptr;
  std::vector<uint32_t> hchunk_in_off, hchunk_out_off;
  std::vector<uint8_t> vlabel_host;   // vertex labels (host copy), empty if none
  std::vector<uint64_t> label_edges;  // edges per label (host copy)
};

// ---------------------------------------------------------------------------
// Traversal control block (device memory, one per launch).
// ---------------------------------------------------------------------------
enum StatIdx {
  ST_W = 0,          // product-edge relaxations (per start vertex)
  ST_N,              // product vertices visited (per start vertex)
  ST_PUSH_LEVELS,
  ST_PULL_LEVELS,
  ST_GROUP_EDGES,    // edges read by top-down levels
  ST_GROUP_ROWS,     // adjacency rows opened by top-down levels
  ST_GROUP_VERTICES, // lane-group product vertices discovered
  ST_PULL_EDGES,     // in-edges read by bottom-up levels
  ST_PULL_VERTICES,  // (vertex, state) words examined bottom-up
  ST_ALG_BYTES,      // algorithmic bytes of the traversal (see the kernel)
  ST_GROUP_W,        // W_g: out-degree over the state's labels, summed over lane-group product vertices
  ST_GROUP_X,        // X_g: (label) adjacency rows of lane-group product vertices
  ST_COUNT
};

constexpr int TRACE_LEVELS = 64;
constexpr unsigned long long NO_ENTRY = ~0ull;      // a reserved list slot left empty
constexpr unsigned int ERR_LIST_OVERFLOW = 1000u;   // BfsCtl::err: an append ran past list_cap
constexpr unsigned int APPEND_SEG = 128;             // list slots a warp reserves at a time

struct BfsCtl {
  unsigned int bar_count;
  unsigned int bar_gen;
  unsigned int err;
  unsigned int err_where;
  unsigned long long n_list[3];
  unsigned long long cursor[3];
  unsigned long long mf[3];
  unsigned long long spill_count[3];   // top-down row chunks queued this level
  unsigned long long spill_cursor[3];
  unsigned long long heavy_cursor[3];  // bottom-up row chunks taken
  unsigned int smask[3];               // DFA states present in each frontier
  unsigned long long levels;
  unsigned long long stats[ST_COUNT];
  // per-level trace (first TRACE_LEVELS levels): start time (ns), frontier
  // entries, direction (1 top-down, 2 bottom-up)
  unsigned long long trace_t[TRACE_LEVELS + 1];
  unsigned long long trace_n[TRACE_LEVELS];
  unsigned int trace_mode[TRACE_LEVELS];
  unsigned long long trace_mf[TRACE_LEVELS];  // frontier out-edges (top-down cost)
  unsigned long long trace_c[TRACE_LEVELS];   // start time (ns) of each level's commit phase
};

// A top-down row longer than SPILL_EDGES is cut into chunks of SPILL_EDGES
// edges that all warps share in a sub-phase of the level.
constexpr unsigned int SPILL_EDGES = 1024;
constexpr unsigned long long SPILL_CAP = 1ull << 18;  // chunks per level

struct BfsParams {
  // graph
  const uint32_t *out_off;
  const uint32_t *out_col;
  const uint32_t *in_off;
  const uint32_t *in_col;
  const uint32_t *hchunk;       // chunks of long in_off rows (nullptr: none)
  uint32_t hchunk_off[RPQ_MAX_LABELS + 1];
  unsigned long long label_edges[RPQ_MAX_LABELS];
  uint32_t n;
  uint32_t L;             // edge labels of the graph
  // lane groups
  uint32_t G;             // groups in this launch
  uint32_t Q;             // DFA states
  const uint32_t *lanesrc;  // [G * 64 * NW], 0xFFFFFFFF = empty lane
  // workspace
  unsigned long long *vis;     // [Q][n][G][NW]: groups innermost
  unsigned long long *fr0;     // frontier ping
  unsigned long long *fr1;     // frontier pong
  unsigned int *claim;         // [Q][n][G] level stamps (NW > 1)
  unsigned long long *spill;   // SPILL_CAP chunk records (nullptr: no spilling)
  unsigned long long spill_cap;  // records usable per level (<= SPILL_CAP)
  unsigned long long *list0;   // entries ((g*Q+q) << 32 | v)
  unsigned long long *list1;
  // Optional frontier bitmaps (nullptr: none), two of fbits_words words: bit
  // q*n + v of bitmap (level & 1) is set when some group holds (q, v) in the
  // level's frontier; bottom-up levels over a sparse frontier test it before
  // gathering a neighbour's frontier words.  Zero between searches.
  unsigned int *fbits;
  unsigned long long fbits_words;
  // List appends: a warp reserves append_seg slots at a time (0: one atomic
  // add per warp-aggregated append); unused reserved slots hold NO_ENTRY.
  unsigned int append_seg;
  unsigned long long list_cap;  // entries per list (overflow sets ERR_LIST_OVERFLOW)
  // Per-group automata (multi mode; nullptr otherwise): group g runs qg[g].
  // q is then the union of the groups' automata over states 0 .. Q-1: it
  // drives the bottom-up iteration and the cost estimates, while qg[g] drives
  // group g's top-down steps and work counters and from_tab[(g * Q + q2) * L
  // + l] is the set of group g's states that reach q2 on label l.
  const QueryDesc *qg;
  const unsigned int *from_tab;
  // Per-lane automata (lane mode; nullptr otherwise): every lane runs its own
  // minimal DFA (states 0 .. Q_i - 1, start state 0).  q then holds the union
  // of the lanes' automata in its bottom-up form (in_begin / in_label /
  // in_from over states 0 .. Q - 1): it drives bottom-up iteration and the
  // cost estimates.  The union's transitions (state, label, target) are listed
  // per source state: transition t of state s is la_trans[t] for
  // la_out_begin[s] <= t < la_out_begin[s + 1], the label in the low 16 bits
  // and the target above; la_mask[t * G * NW + g * NW + k] holds the lanes of
  // word k of group g that take it.  la_in_t[j * Q + s] is the transition
  // from state s of bottom-up group j (the group's label into its target).
  const unsigned short *la_out_begin;
  const unsigned int *la_trans;
  const unsigned long long *la_mask;
  const unsigned short *la_in_t;
  // the union's transitions grouped by (state, label): groups la_grp_begin[q]
  // .. la_grp_begin[q + 1] of state q, la_grp[i] = label | (transitions << 16),
  // la_gmask[i * G * NW ..] the OR of the group's lane masks (a lane's own DFA
  // takes at most one transition per (state, label), so the masks are disjoint)
  const unsigned short *la_grp_begin;
  const unsigned int *la_grp;
  const unsigned long long *la_gmask;
  BfsCtl *ctl;
  unsigned int stamp_base;     // claim stamps continue across launches
  unsigned int nblocks;
  unsigned int pull_dynamic;   // bottom-up levels take vertex chunks from a cursor (else round-robin)
  unsigned int lane_by_source; // lane mode: light bottom-up rows gathered once per (label, source state)
  int force;                   // 0 auto, 1 push only, 2 pull only
  float alpha;                 // push if alpha * push_cost < pull_cost
  unsigned long long time_limit_ns;
  QueryDesc q;
};

// Launchers (return cudaError_t of the launch).
cudaError_t launch_vis_init(int nw, const BfsParams &p, const unsigned long long *empty, cudaStream_t st);
cudaError_t launch_msbfs(int nw, const BfsParams &p, int blocks, int threads, cudaStream_t st);
// Per-group automata (p.qg set): one lane word per group (NW = 1).
cudaError_t launch_msbfs_multi(const BfsParams &p, int blocks, int threads, cudaStream_t st);
int msbfs_multi_max_blocks(int threads, int *blocks_per_sm);
// Per-lane automata (p.la_* set), NW = 1 or 4.  VIS starts as empty_q[(q * G +
// g) * NW + k]: the lanes that are empty or whose automaton has no state q.
cudaError_t launch_msbfs_lane(int nw, const BfsParams &p, int blocks, int threads, cudaStream_t st);
int msbfs_lane_max_blocks(int nw, int threads, int *blocks_per_sm);
cudaError_t launch_vis_init_lane(int nw, const BfsParams &p, const unsigned long long *empty_q, cudaStream_t st);
// flag[i] = whether srcs[i] has an edge (offsets `off`, per label) on a label of label_mask.
cudaError_t launch_source_filter(const uint32_t *off, uint32_t n, uint32_t L, unsigned long long label_mask,
                                 const uint32_t *srcs, unsigned long long count, unsigned char *flag,
                                 cudaStream_t st);
int msbfs_max_blocks(int nw, int threads, int *blocks_per_sm, int *sms);

struct EmitParams {
  const unsigned long long *vis;
  uint32_t n;
  uint32_t G;
  uint32_t Q;
  uint32_t final_mask;
  const uint32_t *lanesrc;
  uint32_t segs;                 // segments per group
  uint32_t *cnt;                 // [G * K][segs]
  const unsigned long long *off; // exclusive offsets of cnt (write pass)
  uint32_t *dst;                 // output destinations (write pass)
  unsigned long long *digest;    // [2]: sum, xor
  const uint32_t *final_g;       // per-group accepting masks (multi mode), else nullptr
  // per-lane accepting lanes (lane mode), else nullptr: word [q * G * NW + g
  // * NW + k] holds the lanes of word k of group g whose automaton accepts in
  // state q (final_mask is then the union of the lanes' accepting states)
  const unsigned long long *final_lane;
  // write pass: lanes whose rows also go out as bitsets over the vertices.
  // lane_slot[lane] = the lane's bitset index (bitset at bits + slot *
  // bwords, bwords a multiple of 4), NO_SOURCE for none; nullptr: no
  // bitsets.  With keep_lists = 0 such lanes write no destinations (their
  // counts must have been zeroed before the offsets were scanned).
  const uint32_t *lane_slot;
  unsigned long long *bits;
  uint64_t bwords;
  uint32_t keep_lists;
};
constexpr int EMIT_TILES = 128;  // 32-vertex tiles per segment
constexpr int EMIT_SEG = 32 * EMIT_TILES;
cudaError_t launch_emit(int nw, bool write, bool digest, const EmitParams &p, cudaStream_t st);
// Digest (sum, xor of splitmix64(src << 32 | dst)) of a materialized chunk's
// rows, added into digest[0..1].
cudaError_t launch_row_digest(const uint32_t *lanesrc, const unsigned long long *lane_off, uint32_t n_lanes,
                              const uint32_t *dst, unsigned long long *digest, cudaStream_t st);
// Per-lane row count and digest (lane_stats[3 * lane + {0, 1, 2}] = rows,
// digest sum, digest xor over the lane's (source, y) rows); lane_stats zeroed
// by the caller.
cudaError_t launch_emit_lane_stats(int nw, const EmitParams &p, unsigned long long *lane_stats, cudaStream_t st);

// Write pass into interleaved (src, dst) rows of a caller's buffer (NW = 1).
cudaError_t launch_emit_pairs(const EmitParams &p, uint32_t *out, cudaStream_t st);

// Load (under the runtime's lazy module loading) the kernels the entry point
// that allocates nothing launches, so that their first use allocates nothing.
cudaError_t preload_static_msbfs_kernels();
cudaError_t preload_static_emit_kernels();
cudaError_t preload_scan_kernels();

// cnt[lane][*] = 0 for every lane with lane_slot[lane] != NO_SOURCE.
cudaError_t launch_zero_lane_counts(uint32_t *cnt, uint32_t segs, uint32_t n_lanes, const uint32_t *lane_slot,
                                    cudaStream_t st);
cudaError_t launch_gather_lane_off(const unsigned long long *off, uint32_t segs, uint32_t n_lanes,
                                   const unsigned long long *total, unsigned long long *lane_off, cudaStream_t st);

// Pair expansion for fetch: out[2k], out[2k+1] = (src, dst) of row first + k.
cudaError_t launch_expand_pairs(const uint32_t *lanesrc, const unsigned long long *lane_off, uint32_t n_lanes,
                                const uint32_t *dst, unsigned long long first, unsigned long long count,
                                uint32_t *out, cudaStream_t st);

// Device-wide exclusive scans.  `tmp` must hold scan_tmp_words(n) words.
size_t scan_tmp_words(size_t n);
cudaError_t exclusive_scan_u32_to_u64(const uint32_t *in, unsigned long long *out, size_t n,
                                      unsigned long long *total, unsigned long long *tmp, cudaStream_t st);
cudaError_t exclusive_scan_u64(const unsigned long long *in, unsigned long long *out, size_t n,
                               unsigned long long *total, unsigned long long *tmp, cudaStream_t st);

// Start-in-the-middle plan: (src, dst, label) triples of the out-CSR (triple
// e = out_col index e), and of a materialized chunk's rows with label x from
// position base.
cudaError_t launch_csr_triples(const uint32_t *off, const uint32_t *col, uint32_t n, uint32_t L, uint32_t *src,
                               uint32_t *dst, uint16_t *lab, cudaStream_t st);
cudaError_t launch_chunk_triples(const uint32_t *lanesrc, const unsigned long long *lane_off, uint32_t n_lanes,
                                 const uint32_t *cdst, unsigned long long base, uint16_t x, uint32_t *src,
                                 uint32_t *dst, uint16_t *lab, cudaStream_t st);

// Graph construction.  Returns RPQ_OK or an error code with *msg set.
int build_graph(DevGraph *g, uint32_t n, uint32_t L, uint64_t m, const uint32_t *d_src, const uint32_t *d_dst,
                const uint16_t *d_lab, cudaStream_t st, std::string *msg);
int graph_key_bits(uint32_t n, uint32_t L);

// Stable LSD radix sort of 64-bit keys over bits [lo_bit, hi_bit); the result
// is in *a afterwards (the two buffers are swapped as needed).
cudaError_t sort_keys_u64(unsigned long long **a, unsigned long long **b, size_t m, int lo_bit, int hi_bit,
                          cudaStream_t st);
// Distinct keys of a sorted array, in order; *d_count (device) gets their number.
cudaError_t unique_keys_u64(const unsigned long long *sorted, size_t m, unsigned long long *out,
                            unsigned long long *d_count, cudaStream_t st);

}  // namespace rpq
