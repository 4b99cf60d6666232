/*
 * rpq.h -- C ABI of the GB300 regular path query engine.
 *
 * The engine evaluates regular path queries (RPQs) and conjunctive regular
 * path queries (CRPQs) over a labeled directed graph resident in GPU memory,
 * following the problem statement of cuRPQ (arXiv 2602.20748):
 *
 *   * Data graph G = (V, E, L), directed, with vertex and edge labels
 *     (Section 2.1).  Vertices are 0 .. n_vertices-1; an edge is a
 *     (src, dst, label) triple; identical triples count once; self-loops are
 *     kept; edges with the same endpoints and different labels are distinct.
 *   * RPQ x -rho-> y (Definition 1): the set of distinct pairs (x, y) joined
 *     by a directed path whose label word is in L(rho).  Paths of any length,
 *     including length 0 when the empty word is in L(rho) (then (v, v) is a
 *     result for every start vertex v).
 *   * CRPQ (Definition 2): all maps f from query variables to vertices such
 *     that labeled variables map to vertices with that label and every atom
 *     x -rho-> y holds for (f(x), f(y)).  Homomorphism (not injective)
 *     semantics, set results.
 *
 * Evaluation is the automata-based method of Section 2.2: a traversal of the
 * product of G with the query automaton (here a minimal DFA), with a visited
 * set per start vertex.  All traversal, deduplication, emission and join work
 * runs in CUDA kernels on the device; the host parses the regex and drives
 * batches.
 *
 * Conventions for every function:
 *   * Return RPQ_OK (0) on success or a negative RPQ_ERR_* code.  On error
 *     the out-pointer is left NULL and rpq_last_error(ctx) describes the
 *     failure (for PARSE errors it contains the byte position).
 *   * Input arrays are host pointers, read during the call and never kept:
 *     the caller keeps ownership.  Handles (rpq_graph, rpq_query, rpq_result)
 *     are owned by the caller after creation and are released with the
 *     matching free_* function, before or after rpq_destroy of their context.
 *   * Result rows are distinct and sorted ascending lexicographically as
 *     unsigned 32-bit values: (src, dst) for an RPQ, the variables in
 *     declaration order for a CRPQ.
 *   * A context is not thread-safe; calls on one context are serialized by
 *     the caller.  All device work of a context is ordered on its stream.
 */
#ifndef GB300_RPQ_H
#define GB300_RPQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes -------------------------------------------------------- */
#define RPQ_OK 0
#define RPQ_ERR_INVALID_ARG -1   /* NULL pointer, id out of range, bad size  */
#define RPQ_ERR_PARSE -2         /* regex syntax error                       */
#define RPQ_ERR_UNKNOWN_LABEL -3 /* regex names a label not in the table     */
#define RPQ_ERR_TOO_COMPLEX -4   /* automaton beyond the engine's limits     */
#define RPQ_ERR_OUT_OF_BUDGET -5 /* device memory budget exceeded            */
#define RPQ_ERR_CUDA -6          /* a CUDA runtime call failed               */
#define RPQ_ERR_TIMEOUT -7       /* a device-side wait ran out of time       */
#define RPQ_ERR_NO_DEVICE -8     /* context has no GPU (host-only context)   */
#define RPQ_ERR_CANCELLED -9     /* server request cancelled before it ended */

/* ---- limits ------------------------------------------------------------- */
#define RPQ_MAX_LABELS 64      /* edge labels per graph                      */
#define RPQ_MAX_STATES 32      /* states of the minimal DFA of one regex     */
#define RPQ_MAX_POSITIONS 63   /* label occurrences in one regex             */
#define RPQ_MAX_TRANSITIONS 256
#define RPQ_MAX_VARS 8         /* CRPQ variables                             */
#define RPQ_MAX_ATOMS 16       /* CRPQ atoms                                 */

/* ---- flags for run_rpq / run_rpq_range / run_crpq ------------------------ */
#define RPQ_MATERIALIZE 0x1u   /* keep result rows on the device (fetch_pairs) */
#define RPQ_COUNT_ONLY 0x2u    /* count rows and digest them; keep no rows    */
#define RPQ_REVERSE 0x4u       /* evaluate from the target end (see run_rpq)  */
#define RPQ_PER_QUERY 0x8u     /* run_rpq_batch: a row count and digest per
                                  query (result_query_stats); no rows kept    */
#define RPQ_FORCE_PUSH 0x100u  /* every level expands top-down (testing)      */
#define RPQ_FORCE_PULL 0x200u  /* every level expands bottom-up (testing)     */

typedef struct rpq_ctx rpq_ctx;
typedef struct rpq_graph rpq_graph;
typedef struct rpq_query rpq_query;
typedef struct rpq_result rpq_result;

/* ---- context ------------------------------------------------------------ */

/* Creates a context on CUDA device `device`.  `mem_budget_bytes` caps the
 * device memory the context allocates for graphs, traversal workspace and
 * results (0: 90% of the device memory free at creation).  `cuda_stream` is
 * a cudaStream_t on that device on which all work is issued (NULL: the
 * legacy default stream).  device = -1 creates a host-only context on which
 * only compile_rpq / query_info work (for tooling without a GPU).
 * Errors: INVALID_ARG (out == NULL), CUDA (device unavailable). */
int rpq_create(rpq_ctx **out, int device, uint64_t mem_budget_bytes, void *cuda_stream);

/* Waits for the context's stream and releases its workspace.  If graphs or
 * results made with the context are still alive, the release is deferred
 * until the last of them is freed (so handles may be freed in any order);
 * the context must not be used for new work after this call.  NULL is
 * ignored. */
void rpq_destroy(rpq_ctx *ctx);

/* Text of the last error on this context ("" if none).  Valid until the next
 * call on the context.  ctx == NULL gives the last error of rpq_create. */
const char *rpq_last_error(const rpq_ctx *ctx);

/* Replaces the stream all later work is issued on (NULL: default stream). */
int rpq_set_stream(rpq_ctx *ctx, void *cuda_stream);

/* Sets a tunable of the context (0 on success, INVALID_ARG for an unknown
 * name or a value out of range):
 *   "alpha"        top-down is chosen for a level when alpha * its bytes are
 *                  below the bottom-up bytes (default 16)
 *   "lane_alpha"   the same for lane-mode launches (one automaton per lane;
 *                  default 2)
 *   "pull_dynamic" 1 (default): bottom-up levels take chunks of 32 vertices
 *                  from a shared cursor; 0: warp k takes chunks k, k + warps,
 *                  ... (same results)
 *   "lane_by_source" 1 (default): bottom-up levels of lane-mode launches
 *                  whose union automaton has at most 8 states gather a
 *                  neighbour's frontier words once per (label, source state)
 *                  and mask them into every target state; 0: once per union
 *                  transition (same results)
 *   "crpq_bitset_frac" run_crpq: an atom's row with at least this fraction
 *                  of the vertices among its destinations is also written as
 *                  a bitset over the vertices, so that a membership test in
 *                  it is one load instead of a binary search; in the last
 *                  step of a count-only CRPQ such rows are kept as bitsets
 *                  only, and a partial tuple whose rows are all bitsets is
 *                  extended by a word-by-word AND of them.  0 .. 2 (default
 *                  1/64: the bitset is at most twice the row's list; 0: every
 *                  non-empty row; above 1: none).  Bitsets take at most half
 *                  of the budget left, longest rows first.
 *   "grid_share"   fraction (0, 1] of the SMs the persistent traversal grids
 *                  occupy (default 1; 0.5 lets two contexts' searches run
 *                  side by side)
 *   "max_groups"   lane groups (256 start vertices each) per launch, 1 .. 16
 *   "time_limit_s" bound on each device-side wait (default 20 s)
 *   "batch_evict"  run_rpq_batch with RPQ_PER_QUERY: product vertices after
 *                  which a query leaves the shared launch (0: never)
 *   "batch_streams" helper contexts evaluating evicted queries side by
 *                  side, 1 .. 16 (default 4)
 *   "batch_lanes"  run_rpq_batch with RPQ_PER_QUERY: evicted queries run in
 *                  lane-mode launches of up to this many lanes, one automaton
 *                  per lane, 1 .. 4096 (default 4096); 0: one bit-sliced
 *                  launch per distinct automaton instead
 *   "batch_direct" 1: every query of such a batch goes straight to the
 *                  lane-mode launches (no shared per-query launch first)
 *   "batch_hash"   1: the shared per-query launch keeps an open-addressing
 *                  visited set (and result set) of 2 x batch_evict slots per
 *                  query instead of dense per-state bitmaps; rows are counted
 *                  as they are found, and a full table evicts its query
 *   "batch_multi"  with batch_lanes = 0: evicted queries of small automaton
 *                  groups share multi-automaton launches
 * A server's workers take the tunables of the context it was created on. */
int rpq_set_option(rpq_ctx *ctx, const char *name, double value);
/* Reads a tunable set by rpq_set_option or chosen by rpq_autotune_batch
 * (same names, plus "batch_threads" and "batch_queries_per_launch"). */
int rpq_get_option(const rpq_ctx *ctx, const char *name, double *value);

/* ---- graph store (Section 2.1 data graph; Section 2.4 keeps one grid per
 *      edge label -- here one CSR per edge label) ----------------------------- */

/* Copies n_edges (src[i], dst[i], label[i]) triples to the device, removes
 * identical triples and builds per-label out- and in-adjacency (CSR, 32-bit
 * ids) resident in device memory.  vertex_label (n_vertices bytes) may be
 * NULL.  Requires n_vertices < 2^31, n_labels in 1 .. RPQ_MAX_LABELS,
 * n_edges < 2^32; every id and label in range.
 * Errors: INVALID_ARG, OUT_OF_BUDGET, CUDA. */
int load_graph(rpq_ctx *ctx, uint32_t n_vertices, uint32_t n_labels, uint64_t n_edges, const uint32_t *src,
               const uint32_t *dst, const uint16_t *label, const uint8_t *vertex_label, rpq_graph **out);

/* Sizes of a loaded graph; n_edges counts distinct triples.  Any out pointer
 * may be NULL. */
int graph_info(const rpq_graph *g, uint32_t *n_vertices, uint32_t *n_labels, uint64_t *n_edges);

void free_graph(rpq_graph *g);

/* ---- query compilation (Section 2.2 automata-based plan; Section 4.1 uses the
 *      minimal DFA of the expression) --------------------------------------- */

/* Parses `regex` and builds its minimal DFA on the host.
 * Syntax: '|' alternation, postfix '*', '+', '?', concatenation by '.',
 * U+00B7 (middle dot, UTF-8) or juxtaposition, parentheses, blanks ignored.
 * With label_names == NULL a label is one lowercase letter, 'a' = 0 ...
 * 'z' = 25.  Otherwise a label is a maximal identifier [A-Za-z0-9_]+ whose
 * index in label_names[0 .. n_names-1] is its label id.  Label ids at or
 * above a graph's n_labels are legal and match no edge of that graph.
 * Errors: INVALID_ARG, PARSE, UNKNOWN_LABEL, TOO_COMPLEX (more than
 * RPQ_MAX_POSITIONS label occurrences, RPQ_MAX_STATES DFA states, or
 * RPQ_MAX_TRANSITIONS transitions, or a label id >= RPQ_MAX_LABELS). */
int compile_rpq(rpq_ctx *ctx, const char *regex, const char *const *label_names, uint32_t n_names,
                rpq_query **out);

/* The compiled minimal DFA: state 0 is the start state; bit q of *final_mask
 * marks accepting states; next[q * n_labels_out + l] is the target of label l
 * from state q or -1.  `next` may be NULL (then only sizes are returned); it
 * must hold n_states * n_labels_out entries, where n_labels_out = (largest
 * label id used) + 1.  Any other out pointer may be NULL. */
int query_info(const rpq_query *q, uint32_t *n_states, uint32_t *n_labels_out, uint64_t *final_mask,
               int32_t *next);

void free_query(rpq_query *q);

/* ---- RPQ evaluation (Definition 1; Section 2.2 product-graph traversal) ---- */

/* Single-source / multi-source RPQ: the result pairs (s, y) for every s in
 * sources[0 .. n_sources-1] (duplicates ignored).  sources == NULL with
 * n_sources == 0 means every vertex (all-pairs).  flags: exactly one of
 * RPQ_MATERIALIZE or RPQ_COUNT_ONLY, optionally one RPQ_FORCE_* (testing).
 * With RPQ_REVERSE the listed vertices are targets instead: the rows are the
 * pairs (y, x) with x -rho-> y for every listed y, found by traversing
 * in-edges with the minimal DFA of the reversed language (the reverse plan
 * of Section 2.3 / the in-edge direction of Section 6.3); sorted by y, x.
 * Errors: INVALID_ARG (source out of range, bad flags), OUT_OF_BUDGET,
 * CUDA, TIMEOUT, TOO_COMPLEX (RPQ_REVERSE and the reversed language needs
 * more than RPQ_MAX_STATES states). */
int run_rpq(rpq_ctx *ctx, const rpq_graph *g, const rpq_query *q, const uint32_t *sources, uint32_t n_sources,
            uint32_t flags, rpq_result **out);

/* All-pairs restricted to the start vertices src_begin <= s < src_end (one
 * batch of an all-pairs evaluation; batches in increasing order concatenate
 * to the sorted all-pairs result).  Same flags and errors as run_rpq. */
int run_rpq_range(rpq_ctx *ctx, const rpq_graph *g, const rpq_query *q, uint32_t src_begin, uint32_t src_end,
                  uint32_t flags, rpq_result **out);

/* ---- start-in-the-middle plan (Section 2.3 WavePlan, plan A3, executed as
 *      A5 of Section 6.3: a sub-RPQ materialized, then joined) ------------- */

/* Evaluates rho = alpha . beta (concatenation) from the listed start vertices
 * (NULL / 0: all-pairs) by starting in the middle: R(beta) is first
 * evaluated and materialized from every vertex at which an alpha path can
 * end (every vertex if the empty word is in L(alpha), else those with an
 * in-edge on a label entering an accepting state of alpha); its pairs
 * become the edges of one extra label X of a temporary graph beside G's own
 * edges; then alpha . X is evaluated over that graph by the ordinary
 * traversal.  The result is the same relation as run_rpq of alpha . beta
 * (Definition 1) -- the plan only changes the order of exploration.  flags:
 * RPQ_MATERIALIZE or RPQ_COUNT_ONLY (optionally RPQ_FORCE_*).  result_stats
 * counts the work of both phases (it differs from the forward plan's W).
 * Device memory: R(beta) is held once as rows and once as a graph label.
 * Errors: INVALID_ARG, OUT_OF_BUDGET, TOO_COMPLEX (the graph already uses
 * RPQ_MAX_LABELS labels, or G's edges plus R(beta) exceed 2^32), CUDA,
 * TIMEOUT. */
int run_rpq_middle(rpq_ctx *ctx, const rpq_graph *g, const rpq_query *alpha, const rpq_query *beta,
                   const uint32_t *sources, uint32_t n_sources, uint32_t flags, rpq_result **out);

/* ---- batched single-source RPQs (many expressions, one launch) ----------- */

/* Evaluates n_queries single-source RPQs together: query i is the compiled
 * expression queries[i] (different queries may use different expressions)
 * from the start vertex sources[i] (host arrays).  All queries advance level
 * by level in one persistent traversal launch (several launches when they
 * do not fit the device together).  Rows are (i, y) for every y with
 * sources[i] -rho_i-> y, sorted by i then y; arity 2.  The digest of
 * result_info is taken over these (i, y) rows.  flags: RPQ_MATERIALIZE or
 * RPQ_COUNT_ONLY, or RPQ_PER_QUERY: every query's own rows (sources[i], y)
 * are counted and digested as run_rpq(queries[i], {sources[i]}) would report
 * them (result_query_stats), and result_info totals those summaries.  In
 * that mode a query whose product graph grows past a threshold (option
 * "batch_evict", product vertices; default 65,536) leaves the shared launch,
 * and such queries are then evaluated together by the multi-source engine in
 * lane-mode launches: one bit lane per query, each lane with its own
 * automaton (option "batch_lanes"; "batch_direct" sends every query there).
 * result_query_time gives each query's completion time.
 * Block size, queries per launch and the threshold come from the last
 * rpq_autotune_batch on the context (defaults otherwise).
 * Errors: INVALID_ARG, OUT_OF_BUDGET, CUDA, TIMEOUT. */
int run_rpq_batch(rpq_ctx *ctx, const rpq_graph *g, uint32_t n_queries, const rpq_query *const *queries,
                  const uint32_t *sources, uint32_t flags, rpq_result **out);

/* Times run_rpq_batch (RPQ_PER_QUERY) on a sample of the given batch (its
 * first 1,024 queries) for each candidate visited-set representation and
 * schedule -- every query straight to lane-mode launches (bit-sliced visited
 * words, one automaton per lane), or a shared per-query launch first with
 * dense bitmaps or open-addressing hash tables, block size 256 or 512 and
 * eviction threshold 2^10, 2^12 or 2^14 product vertices, the evicted
 * queries then in lane-mode launches -- keeps the fastest on the context for
 * later run_rpq_batch calls (options batch_direct, batch_hash, batch_evict,
 * batch_threads) and reports it (out pointers may be NULL; queries per launch
 * is reported as set).
 * Errors: as run_rpq_batch. */
int rpq_autotune_batch(rpq_ctx *ctx, const rpq_graph *g, uint32_t n_queries, const rpq_query *const *queries,
                       const uint32_t *sources, uint32_t *threads_out, uint32_t *queries_per_launch_out);

/* ---- RPQ evaluation that allocates no device memory ---------------------- */

/* The paper has no counterpart to this entry point.  It serves callers that
 * cannot allocate device memory while they query: an application that gives
 * the whole device memory to its own pool or buffer manager at start-up, a
 * latency-critical loop that must not take the device-wide synchronization
 * an allocation may imply, or code hosted inside another runtime that
 * forbids allocating on its device.  It evaluates the same RPQ as run_rpq for
 * 1 .. 64 start vertices, but every byte of scratch it uses lives in one
 * 64 MiB array per device that the library reserves when the first context on
 * that device is created (rpq_create looks up the array's device address with
 * cudaGetSymbolAddress, which loads it, and loads the kernels this call
 * launches) and keeps until the process exits; the call itself calls no
 * cudaMalloc, cudaFree or other allocating routine.  A context created after
 * a cudaDeviceReset looks the address up again.
 *   sources    host array of n_sources start vertices (duplicates ignored).
 *   out_pairs  caller-owned DEVICE buffer of 2 * max_rows uint32 values; row
 *              k is written as (src, dst) at out_pairs[2k], out_pairs[2k+1],
 *              rows sorted as for run_rpq.
 *   *n_rows    (host) the number of result rows.
 * The graph and query must fit the array: about 40 * states * vertices bytes
 * (plus a little per 1,024 vertices); larger ones are rejected with
 * OUT_OF_BUDGET and a message naming both sizes.  If the result has more than
 * max_rows rows, nothing is written, *n_rows holds the row count and the call
 * returns OUT_OF_BUDGET.  All calls share the array, and each keeps the
 * previous call's contents until it clears what it needs: calls whose GPU
 * work overlaps (from several threads or streams on one device) race and
 * must be serialized by the caller.  The call waits for its work to finish.
 * Errors: INVALID_ARG (NULL pointer, n_sources not in 1 .. 64, a source out of
 * range), NO_DEVICE, OUT_OF_BUDGET, CUDA (a CUDA call failed, or the
 * traversal's entry list overflowed -- an internal error), TIMEOUT (a
 * traversal barrier wait ran out of time). */
int run_rpq_static(rpq_ctx *ctx, const rpq_graph *g, const rpq_query *q, const uint32_t *sources,
                   uint32_t n_sources, uint32_t *out_pairs, uint64_t max_rows, uint64_t *n_rows);

/* ---- CRPQ evaluation (Definition 2; Section 6.3 joins atom results) ------- */

typedef struct {
  uint32_t x;         /* source variable index                             */
  uint32_t y;         /* target variable index                             */
  const rpq_query *q; /* the atom's compiled regex                         */
} crpq_atom;

/* Evaluates a CRPQ with n_vars variables (1 .. RPQ_MAX_VARS) and n_atoms
 * atoms (1 .. RPQ_MAX_ATOMS).  var_label[i] >= 0 requires f(i) to carry that
 * vertex label (needs a graph loaded with vertex labels); -1 or a NULL array
 * means no constraint.  Every variable must occur in some atom, and the
 * atoms must connect all variables.  restrict0 (may be NULL) limits
 * variable 0 to the listed vertices -- a batch of the full query.  Rows are
 * n_vars-tuples in declaration order.  flags as for run_rpq.  Variables are
 * bound one at a time (values of variable 0 in batches of 4,096); each atom
 * is evaluated from the distinct values its bound end takes, and its long
 * rows are also held as bitsets over the vertices (option
 * "crpq_bitset_frac").  With RPQ_COUNT_ONLY the last variable (unless an
 * atom loops on it) is bound, counted and digested in one pass, without
 * materializing tuples.
 * Errors: INVALID_ARG, OUT_OF_BUDGET, CUDA, TIMEOUT. */
int run_crpq(rpq_ctx *ctx, const rpq_graph *g, uint32_t n_vars, const int32_t *var_label, const crpq_atom *atoms,
             uint32_t n_atoms, const uint32_t *restrict0, uint32_t n_restrict0, uint32_t flags,
             rpq_result **out);

/* ---- serving: continuous batching of mixed requests ----------------------- */

/* A server evaluates RPQ and CRPQ requests that arrive over time against one
 * resident graph, with continuous batching.  Single-source requests enter a
 * persistent serving launch through a ring in mapped host memory: at every
 * BFS level boundary the launch admits as many waiting requests as it has
 * free slots for (each slot holds one query's open-addressing visited set
 * and result set, so admission is bounded by that device memory; max_batch
 * caps the slots), and a query leaves its slot the level its frontier runs
 * empty, with its row count and digest already accumulated, so requests that
 * arrive while others are on the device join them and finish on their own
 * schedule.  A query that grows past 4,096 product vertices leaves the launch
 * and is finished, with every other such query waiting, in lane-mode
 * launches (one automaton per bit lane).  All-pairs requests and CRPQs run on
 * two bulk workers; each starts the oldest such request once its estimated
 * device memory (traversal state, entry lists, emission scratch, sized by
 * the lane groups it will use) fits what the running bulk requests leave of
 * the bulk share of the budget.  The three kinds of work have their own
 * streams and shares of the SMs, so they overlap on the device.  Replies
 * carry the row count and digest the standalone call would report (results
 * are counted, not kept) and the request's latencies.  The graph, queries
 * and atom queries must stay alive until their requests have been waited
 * for.  mem_budget_bytes = 0 uses 80% of the free device memory. */
typedef struct rpq_server rpq_server;

#define RPQ_REQ_SINGLE 1u   /* rho from one start vertex                    */
#define RPQ_REQ_ALLPAIRS 2u /* rho from every vertex                         */
#define RPQ_REQ_CRPQ 3u     /* a CRPQ (as run_crpq, all values of variable 0) */

typedef struct {
  uint32_t kind;             /* RPQ_REQ_*                                      */
  const rpq_query *q;        /* SINGLE, ALLPAIRS                               */
  uint32_t source;           /* SINGLE                                         */
  uint32_t n_vars;           /* CRPQ                                           */
  const int32_t *var_label;  /* CRPQ, may be NULL; copied at submit            */
  const crpq_atom *atoms;    /* CRPQ; copied at submit                         */
  uint32_t n_atoms;          /* CRPQ                                           */
} rpq_request;

typedef struct {
  int status;                /* RPQ_OK or the evaluation's error code          */
  uint64_t count;            /* result rows                                    */
  uint64_t digest_sum;       /* digest of the rows, as result_info             */
  uint64_t digest_xor;
  double queued_ms;          /* submit -> evaluation start                     */
  double service_ms;         /* evaluation start -> done                       */
  double latency_ms;         /* submit -> done                                 */
} rpq_reply;

int rpq_server_create(rpq_ctx *ctx, const rpq_graph *g, uint64_t mem_budget_bytes, uint32_t max_batch,
                      rpq_server **out);
/* Queues a request; *ticket identifies it for rpq_server_wait. */
int rpq_server_submit(rpq_server *s, const rpq_request *req, uint64_t *ticket);
/* Waits (timeout_s < 0: without limit) for the request and takes its reply;
 * TIMEOUT if it is not done in time (it stays queued). */
int rpq_server_wait(rpq_server *s, uint64_t ticket, double timeout_s, rpq_reply *reply);
/* Serving launches so far and the single-source requests admitted into
 * them (a request that arrives while a launch runs joins it, so launches can
 * be far fewer than requests). */
int rpq_server_stats(rpq_server *s, uint64_t *batches, uint64_t *batched_requests);
/* Counters of a server (all cumulative). */
typedef struct {
  uint64_t launches;       /* serving launches (a new one starts when requests
                              arrive while none is running)                   */
  uint64_t admitted;       /* single-source requests admitted into them       */
  uint64_t lane_requests;  /* of those, finished in lane-mode launches after
                              outgrowing the serving launch                   */
  uint64_t lane_launches;  /* lane-mode launches                              */
  uint32_t graph;          /* 1: serving launches replay a CUDA graph captured
                              at creation; 0: they are issued directly        */
  uint32_t slots;          /* queries the serving launch holds at once        */
} rpq_server_counters;
int rpq_server_info(rpq_server *s, rpq_server_counters *out);
/* Cancels every request not yet done: they complete at once with status
 * RPQ_ERR_CANCELLED (the device finishes single-source requests it has
 * already admitted and drops their replies), and the all-pairs request or
 * CRPQ in service stops before its next launch (next slice of start
 * vertices, next batch of variable-0 values).  The server stays usable. */
int rpq_server_cancel(rpq_server *s);
/* Finishes the queued requests, stops the workers and releases the server. */
void rpq_server_destroy(rpq_server *s);

/* ---- results ------------------------------------------------------------ */

/* Row count, arity (2 for RPQ) and the order-independent digest of the rows:
 * sum (mod 2^64) and xor of h(row) over all rows.  For a row t[0 .. k-1]:
 * k == 1: h = s(t[0]); k >= 2: h = s(t[0] << 32 | t[1]), then for each
 * further column i, h = s(h ^ t[i]).  s(x) is the SplitMix64 output for
 * state x: z = x + 0x9E3779B97F4A7C15, z = (z ^ z >> 30) * 0xBF58476D1CE4E5B9,
 * z = (z ^ z >> 27) * 0x94D049BB133111EB, s = z ^ z >> 31 (mod 2^64).
 * Any out pointer may be NULL. */
int result_info(const rpq_result *r, uint64_t *count, uint32_t *arity, uint64_t *digest_sum,
                uint64_t *digest_xor);

/* Work counters of the evaluation that made the result.  product_edges is
 * the number of product-edge relaxations of a per-start-vertex traversal
 * over the minimal DFA: for every start s, every product vertex (v, q)
 * reachable from (s, q0), every label l leaving q, deg_l(v) -- a measure of
 * the work that does not depend on the engine's design.
 * product_vertices counts the (s, v, q) visited.  The remaining fields
 * describe what the kernels did. */
typedef struct {
  uint64_t product_edges;    /* W                                              */
  uint64_t product_vertices; /* N                                              */
  uint64_t levels;           /* BFS levels summed over lane groups            */
  uint64_t push_levels;      /* levels expanded top-down                      */
  uint64_t pull_levels;      /* levels expanded bottom-up                     */
  uint64_t group_edges;      /* edges read by top-down levels (per lane group) */
  uint64_t group_rows;       /* adjacency rows opened by top-down levels      */
  uint64_t group_vertices;   /* lane-group product vertices discovered        */
  uint64_t pull_edges;       /* in-edges read by bottom-up levels             */
  uint64_t pull_vertices;    /* (vertex, state) words examined bottom-up      */
  uint64_t lane_words;       /* 64-bit words per lane group (1 or 4)          */
  uint64_t lane_groups;      /* lane groups evaluated                         */
  double bfs_ms;             /* device time of the traversal kernels          */
  double emit_ms;            /* device time of the emission kernels           */
  uint64_t bfs_launches;     /* traversal kernel launches                     */
  uint64_t launches;         /* all kernel launches of the evaluation         */
  uint64_t alg_bytes;        /* bytes the traversal kernels must move for the
                                work they did (column ids, offsets, visited and
                                frontier words, list entries)                 */
  uint64_t evicted;          /* run_rpq_batch RPQ_PER_QUERY: queries that left
                                the shared launch                            */
  uint64_t group_product_edges; /* W_g: for every lane-group product vertex
                                   (group, v, q) discovered, deg_l(v) summed
                                   over the labels l leaving q -- the
                                   relaxations one bit-sliced word serves    */
  uint64_t group_label_rows;    /* X_g: adjacency rows (v, l) of those
                                   product vertices (labels present)         */
} rpq_stats;

int result_stats(const rpq_result *r, rpq_stats *out);
/* For a run_rpq_batch result made with RPQ_PER_QUERY: milliseconds from the
 * start of the call until query i's summary was known on the host (queries
 * that finish in the shared launch are known before those evaluated later in
 * lane-mode launches).  INVALID_ARG otherwise or when i is out of range. */
int result_query_time(const rpq_result *r, uint32_t i, double *ms);
/* Row count and digest of query i of a run_rpq_batch result made with
 * RPQ_PER_QUERY (INVALID_ARG otherwise or when i is out of range). */
int result_query_stats(const rpq_result *r, uint32_t i, uint64_t *count, uint64_t *digest_sum, uint64_t *digest_xor);

/* ---- streamed materialization ------------------------------------------- */
/* The rows of rho from start vertices [src_begin, src_end), delivered to the
 * host while the device keeps exploring: the start vertices run in batches of
 * one traversal launch (4,096 sources), and the rows of a finished batch are
 * copied into pinned host memory on a copy stream of the library's own while
 * the next batch's traversal runs -- the batch-wise transfer of results to the
 * host that Section 5 of the paper describes, here with the rows of a block in
 * compressed form (one 4-byte destination per row).  Rows arrive in the order
 * run_rpq_range would list them (ascending (src, dst)).  flags: 0 or
 * RPQ_REVERSE.  The context serves only this stream until rpq_stream_close
 * (the library runs it from two threads of its own); the graph and query must
 * outlive the stream.  Device memory held by rows not yet copied is bounded by
 * four batches; host memory is three pinned slots of 256 MiB, allocated by
 * the first stream on the context and kept by the context for later ones.
 * rpq_stream_open_multi streams several queries over the same range, one
 * after the other (all rows of queries[0], then of queries[1], ...), so that
 * the copies of one query's last batches overlap the next query's first
 * traversals; each block names its query.  The query array is read at open
 * time; the queries themselves must outlive the stream. */
typedef struct rpq_stream rpq_stream;

typedef struct {
  uint32_t n_sources;        /* start vertices with rows in this block        */
  const uint32_t *sources;   /* [n_sources], ascending                        */
  const uint64_t *offsets;   /* [n_sources + 1]: rows of sources[i] are
                                dst[offsets[i] .. offsets[i + 1])             */
  const uint32_t *dst;       /* destinations, ascending per source            */
  uint64_t n_rows;           /* rows in this block; 0 marks the end           */
  uint32_t query;            /* index of the block's query (0 for
                                rpq_stream_open)                              */
} rpq_row_block;

int rpq_stream_open(rpq_ctx *ctx, const rpq_graph *g, const rpq_query *q, uint32_t src_begin, uint32_t src_end,
                    uint32_t flags, rpq_stream **out);
/* n_queries >= 1 queries, none null; INVALID_ARG otherwise. */
int rpq_stream_open_multi(rpq_ctx *ctx, const rpq_graph *g, const rpq_query *const *queries, uint32_t n_queries,
                          uint32_t src_begin, uint32_t src_end, uint32_t flags, rpq_stream **out);
/* Fills *block with the next block of rows.  Its arrays belong to the stream
 * and stay valid until the next rpq_stream_next or rpq_stream_close on it.
 * n_rows = 0 at the end; a failure of the evaluation is returned here (after
 * the blocks that completed before it). */
int rpq_stream_next(rpq_stream *s, rpq_row_block *block);
/* Totals over the batches evaluated so far: rows, row digest, counters. */
int rpq_stream_info(rpq_stream *s, uint64_t *rows, uint64_t *digest_sum, uint64_t *digest_xor, rpq_stats *stats);
void rpq_stream_close(rpq_stream *s);

/* Copies rows [offset, offset + max_rows) (clipped to the row count) into
 * host memory out[arity * k], k rows, and stores k in *n_rows.
 * Requires a result made with RPQ_MATERIALIZE.
 * Errors: INVALID_ARG, CUDA. */
int fetch_pairs(const rpq_result *r, uint64_t offset, uint64_t max_rows, uint32_t *out, uint64_t *n_rows);

void free_result(rpq_result *r);

#ifdef __cplusplus
}
#endif

#endif /* GB300_RPQ_H */
