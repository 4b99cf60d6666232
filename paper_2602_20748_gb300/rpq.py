"""ctypes binding of the C ABI in include/rpq.h (argument marshalling only).

Every computation happens in the CUDA library ``_build/librpq.so``; this
module converts numpy arrays and Python strings to pointers and sizes and
raises :class:`RPQError` on negative return codes.  Importing it fails
loudly when the library has not been built: there is no fallback.

The functions keep the C names (``load_graph``, ``compile_rpq``, ``run_rpq``,
``run_rpq_range``, ``run_crpq``, ``fetch_pairs`` ...).  Handles are wrapped in
small classes whose ``free()`` (also called on garbage collection) calls the
matching ``free_*``.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librpq.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"the CUDA library {LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")

_lib = ctypes.CDLL(LIB_PATH)

RPQ_OK = 0
RPQ_ERR_INVALID_ARG = -1
RPQ_ERR_PARSE = -2
RPQ_ERR_UNKNOWN_LABEL = -3
RPQ_ERR_TOO_COMPLEX = -4
RPQ_ERR_OUT_OF_BUDGET = -5
RPQ_ERR_CUDA = -6
RPQ_ERR_TIMEOUT = -7
RPQ_ERR_NO_DEVICE = -8
RPQ_ERR_CANCELLED = -9

RPQ_MATERIALIZE = 0x1
RPQ_COUNT_ONLY = 0x2
RPQ_REVERSE = 0x4
RPQ_PER_QUERY = 0x8
RPQ_FORCE_PUSH = 0x100
RPQ_FORCE_PULL = 0x200

RPQ_MAX_STATES = 32
RPQ_MAX_LABELS = 64

EXPORTED = [
    "rpq_create", "rpq_destroy", "rpq_last_error", "rpq_set_stream", "load_graph", "graph_info", "free_graph",
    "compile_rpq", "query_info", "free_query", "run_rpq", "run_rpq_range", "run_crpq", "result_info",
    "result_stats", "fetch_pairs", "free_result", "run_rpq_static",
]

c_void_p = ctypes.c_void_p
c_u32 = ctypes.c_uint32
c_u64 = ctypes.c_uint64
P = ctypes.POINTER


class rpq_stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_uint64) for name in (
        "product_edges", "product_vertices", "levels", "push_levels", "pull_levels", "group_edges", "group_rows",
        "group_vertices", "pull_edges", "pull_vertices", "lane_words", "lane_groups")] + [
        ("bfs_ms", ctypes.c_double), ("emit_ms", ctypes.c_double), ("bfs_launches", ctypes.c_uint64),
        ("launches", ctypes.c_uint64), ("alg_bytes", ctypes.c_uint64), ("evicted", ctypes.c_uint64),
        ("group_product_edges", ctypes.c_uint64), ("group_label_rows", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class crpq_atom(ctypes.Structure):
    _fields_ = [("x", c_u32), ("y", c_u32), ("q", c_void_p)]


_lib.rpq_create.argtypes = [P(c_void_p), ctypes.c_int, c_u64, c_void_p]
_lib.rpq_destroy.argtypes = [c_void_p]
_lib.rpq_destroy.restype = None
_lib.rpq_last_error.argtypes = [c_void_p]
_lib.rpq_last_error.restype = ctypes.c_char_p
_lib.rpq_set_stream.argtypes = [c_void_p, c_void_p]
_lib.load_graph.argtypes = [c_void_p, c_u32, c_u32, c_u64, c_void_p, c_void_p, c_void_p, c_void_p, P(c_void_p)]
_lib.graph_info.argtypes = [c_void_p, P(c_u32), P(c_u32), P(c_u64)]
_lib.free_graph.argtypes = [c_void_p]
_lib.free_graph.restype = None
_lib.compile_rpq.argtypes = [c_void_p, ctypes.c_char_p, c_void_p, c_u32, P(c_void_p)]
_lib.query_info.argtypes = [c_void_p, P(c_u32), P(c_u32), P(c_u64), c_void_p]
_lib.free_query.argtypes = [c_void_p]
_lib.free_query.restype = None
_lib.run_rpq.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_u32, c_u32, P(c_void_p)]
_lib.run_rpq_range.argtypes = [c_void_p, c_void_p, c_void_p, c_u32, c_u32, c_u32, P(c_void_p)]
_lib.run_crpq.argtypes = [c_void_p, c_void_p, c_u32, c_void_p, c_void_p, c_u32, c_void_p, c_u32, c_u32,
                          P(c_void_p)]
_lib.result_info.argtypes = [c_void_p, P(c_u64), P(c_u32), P(c_u64), P(c_u64)]
_lib.result_stats.argtypes = [c_void_p, P(rpq_stats)]
_lib.fetch_pairs.argtypes = [c_void_p, c_u64, c_u64, c_void_p, P(c_u64)]
_lib.free_result.argtypes = [c_void_p]
_lib.free_result.restype = None
_lib.run_rpq_static.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_u32, c_void_p, c_u64, P(c_u64)]


class RPQError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rpq error {code}: {msg}")
        self.code = code


def _ptr(a):
    return None if a is None else a.ctypes.data_as(c_void_p)


class Context:
    """rpq_create / rpq_destroy.  ``stream`` is a raw cudaStream_t handle
    (e.g. ``torch.cuda.current_stream().cuda_stream``) or None."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0, stream: int | None = None):
        h = c_void_p()
        rc = _lib.rpq_create(ctypes.byref(h), device, mem_budget_bytes, stream)
        if rc != 0:
            raise RPQError(rc, _lib.rpq_last_error(None).decode())
        self.h = h
        self.device = device

    def check(self, rc: int):
        if rc != 0:
            raise RPQError(rc, _lib.rpq_last_error(self.h).decode())

    def set_stream(self, stream: int | None):
        self.check(_lib.rpq_set_stream(self.h, stream))

    def close(self):
        if getattr(self, "h", None):
            _lib.rpq_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


class Graph:
    def __init__(self, ctx: Context, h):
        self.ctx, self.h = ctx, h

    def info(self):
        n, L, m = c_u32(), c_u32(), c_u64()
        self.ctx.check(_lib.graph_info(self.h, ctypes.byref(n), ctypes.byref(L), ctypes.byref(m)))
        return n.value, L.value, m.value

    def free(self):
        if self.h:
            _lib.free_graph(self.h)
            self.h = None

    def __del__(self):
        self.free()


class Query:
    def __init__(self, ctx: Context, h):
        self.ctx, self.h = ctx, h

    def free(self):
        if self.h:
            _lib.free_query(self.h)
            self.h = None

    def __del__(self):
        self.free()


class Result:
    def __init__(self, ctx: Context, h):
        self.ctx, self.h = ctx, h

    def free(self):
        if self.h:
            _lib.free_result(self.h)
            self.h = None

    def __del__(self):
        self.free()


def load_graph(ctx: Context, n_vertices: int, n_labels: int, src, dst, label, vertex_label=None) -> Graph:
    src = np.ascontiguousarray(src, dtype=np.uint32)
    dst = np.ascontiguousarray(dst, dtype=np.uint32)
    label = np.ascontiguousarray(label, dtype=np.uint16)
    vl = None if vertex_label is None else np.ascontiguousarray(vertex_label, dtype=np.uint8)
    if not (len(src) == len(dst) == len(label)):
        raise ValueError("src, dst and label must have the same length")
    h = c_void_p()
    ctx.check(_lib.load_graph(ctx.h, n_vertices, n_labels, len(src), _ptr(src), _ptr(dst), _ptr(label), _ptr(vl),
                              ctypes.byref(h)))
    return Graph(ctx, h)


def compile_rpq(ctx: Context, regex: str, label_names=None) -> Query:
    h = c_void_p()
    if label_names is None:
        ctx.check(_lib.compile_rpq(ctx.h, regex.encode(), None, 0, ctypes.byref(h)))
    else:
        arr = (ctypes.c_char_p * len(label_names))(*[n.encode() for n in label_names])
        ctx.check(_lib.compile_rpq(ctx.h, regex.encode(), ctypes.cast(arr, c_void_p), len(label_names),
                                   ctypes.byref(h)))
    return Query(ctx, h)


def query_info(q: Query):
    """(n_states, final_mask, next[n_states, n_labels_out]) of the minimal DFA."""
    ns, nl, fm = c_u32(), c_u32(), c_u64()
    q.ctx.check(_lib.query_info(q.h, ctypes.byref(ns), ctypes.byref(nl), ctypes.byref(fm), None))
    nxt = np.full(max(1, ns.value * nl.value), -1, dtype=np.int32)
    q.ctx.check(_lib.query_info(q.h, None, None, None, _ptr(nxt)))
    return ns.value, fm.value, nxt[: ns.value * nl.value].reshape(ns.value, nl.value)


def run_rpq(ctx: Context, g: Graph, q: Query, sources=None, flags: int = RPQ_MATERIALIZE) -> Result:
    h = c_void_p()
    if sources is None:
        ctx.check(_lib.run_rpq(ctx.h, g.h, q.h, None, 0, flags, ctypes.byref(h)))
    else:
        s = np.ascontiguousarray(sources, dtype=np.uint32)
        ctx.check(_lib.run_rpq(ctx.h, g.h, q.h, _ptr(s), len(s), flags, ctypes.byref(h)))
    return Result(ctx, h)


_lib.run_rpq_middle.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_u32, c_u32, P(c_void_p)]
EXPORTED += ["run_rpq_middle"]


def run_rpq_middle(ctx: Context, g: Graph, alpha: Query, beta: Query, sources=None,
                   flags: int = RPQ_MATERIALIZE) -> Result:
    """run_rpq_middle: alpha . beta by the start-in-the-middle plan."""
    s = None if sources is None else np.ascontiguousarray(sources, dtype=np.uint32)
    h = c_void_p()
    ctx.check(_lib.run_rpq_middle(ctx.h, g.h, alpha.h, beta.h, _ptr(s), 0 if s is None else len(s), flags,
                                  ctypes.byref(h)))
    return Result(ctx, h)


def run_rpq_range(ctx: Context, g: Graph, q: Query, src_begin: int, src_end: int,
                  flags: int = RPQ_MATERIALIZE) -> Result:
    h = c_void_p()
    ctx.check(_lib.run_rpq_range(ctx.h, g.h, q.h, src_begin, src_end, flags, ctypes.byref(h)))
    return Result(ctx, h)


def run_crpq(ctx: Context, g: Graph, n_vars: int, atoms, var_label=None, restrict0=None,
             flags: int = RPQ_MATERIALIZE) -> Result:
    """``atoms``: list of (x, Query, y)."""
    arr = (crpq_atom * len(atoms))(*[crpq_atom(a[0], a[2], a[1].h) for a in atoms])
    vl = None if var_label is None else np.ascontiguousarray(var_label, dtype=np.int32)
    r0 = None if restrict0 is None else np.ascontiguousarray(restrict0, dtype=np.uint32)
    h = c_void_p()
    ctx.check(_lib.run_crpq(ctx.h, g.h, n_vars, _ptr(vl), ctypes.cast(arr, c_void_p), len(atoms), _ptr(r0),
                            0 if r0 is None else len(r0), flags, ctypes.byref(h)))
    return Result(ctx, h)


def result_info(r: Result):
    """(count, arity, digest_sum, digest_xor)."""
    n, a, s, x = c_u64(), c_u32(), c_u64(), c_u64()
    r.ctx.check(_lib.result_info(r.h, ctypes.byref(n), ctypes.byref(a), ctypes.byref(s), ctypes.byref(x)))
    return n.value, a.value, s.value, x.value


def result_stats(r: Result) -> dict:
    st = rpq_stats()
    r.ctx.check(_lib.result_stats(r.h, ctypes.byref(st)))
    return st.as_dict()


def fetch_pairs(r: Result, offset: int = 0, max_rows: int | None = None, out: np.ndarray | None = None):
    """Rows [offset, offset + max_rows) as an (k, arity) uint32 array.  ``out``
    may be a preallocated (pinned) uint32 buffer of at least arity*k values."""
    count, arity, _, _ = result_info(r)
    if max_rows is None:
        max_rows = max(0, count - offset)
    k = max(0, min(max_rows, count - offset))
    if out is None:
        out = np.empty(max(1, k * arity), dtype=np.uint32)
    got = c_u64()
    r.ctx.check(_lib.fetch_pairs(r.h, offset, k, _ptr(out), ctypes.byref(got)))
    return out[: got.value * arity].reshape(got.value, arity)


def run_rpq_static(ctx: Context, g: Graph, q: Query, sources, out_pairs_ptr: int, max_rows: int) -> int:
    """run_rpq_static: the RPQ for 1..64 start vertices with no device
    allocation.  ``out_pairs_ptr`` is the address of a caller-owned device
    buffer of 2 * max_rows uint32 values.  Returns the number of rows."""
    s = np.ascontiguousarray(sources, dtype=np.uint32)
    n = c_u64()
    ctx.check(_lib.run_rpq_static(ctx.h, g.h, q.h, _ptr(s), len(s), out_pairs_ptr, max_rows, ctypes.byref(n)))
    return n.value


_lib.run_rpq_batch.argtypes = [c_void_p, c_void_p, c_u32, c_void_p, c_void_p, c_u32, P(c_void_p)]
_lib.rpq_autotune_batch.argtypes = [c_void_p, c_void_p, c_u32, c_void_p, c_void_p, P(c_u32), P(c_u32)]
_lib.result_query_stats.argtypes = [c_void_p, c_u32, P(c_u64), P(c_u64), P(c_u64)]
EXPORTED += ["run_rpq_batch", "rpq_autotune_batch", "result_query_stats"]


_lib.result_query_time.argtypes = [c_void_p, c_u32, P(ctypes.c_double)]
EXPORTED += ["result_query_time"]


def result_query_time(r: Result, i: int) -> float:
    """Milliseconds from the start of run_rpq_batch (RPQ_PER_QUERY) until
    query i's summary was known."""
    ms = ctypes.c_double()
    r.ctx.check(_lib.result_query_time(r.h, i, ctypes.byref(ms)))
    return ms.value


def result_query_stats(r: Result, i: int):
    """(rows, digest sum, digest xor) of query i of a RPQ_PER_QUERY batch."""
    c, s, x = c_u64(), c_u64(), c_u64()
    r.ctx.check(_lib.result_query_stats(r.h, i, ctypes.byref(c), ctypes.byref(s), ctypes.byref(x)))
    return c.value, s.value, x.value


def _query_array(queries):
    return (c_void_p * max(1, len(queries)))(*[q.h.value if isinstance(q.h, c_void_p) else q.h for q in queries])


def run_rpq_batch(ctx: Context, g: Graph, queries, sources, flags: int = RPQ_MATERIALIZE) -> Result:
    """run_rpq_batch: queries[i] (Query) from sources[i]; rows (i, y)."""
    s = np.ascontiguousarray(sources, dtype=np.uint32)
    if len(s) != len(queries):
        raise ValueError("one source per query")
    arr = _query_array(queries)
    h = c_void_p()
    ctx.check(_lib.run_rpq_batch(ctx.h, g.h, len(queries), ctypes.cast(arr, c_void_p), _ptr(s), flags,
                                 ctypes.byref(h)))
    return Result(ctx, h)


def rpq_autotune_batch(ctx: Context, g: Graph, queries, sources):
    """Returns the (threads, queries_per_launch) the autotuner kept."""
    s = np.ascontiguousarray(sources, dtype=np.uint32)
    arr = _query_array(queries)
    t, k = c_u32(), c_u32()
    ctx.check(_lib.rpq_autotune_batch(ctx.h, g.h, len(queries), ctypes.cast(arr, c_void_p), _ptr(s),
                                      ctypes.byref(t), ctypes.byref(k)))
    return t.value, k.value


class rpq_request(ctypes.Structure):
    _fields_ = [("kind", c_u32), ("q", c_void_p), ("source", c_u32), ("n_vars", c_u32), ("var_label", c_void_p),
                ("atoms", c_void_p), ("n_atoms", c_u32)]


class rpq_reply(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("count", c_u64), ("digest_sum", c_u64), ("digest_xor", c_u64),
                ("queued_ms", ctypes.c_double), ("service_ms", ctypes.c_double), ("latency_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


RPQ_REQ_SINGLE = 1
RPQ_REQ_ALLPAIRS = 2
RPQ_REQ_CRPQ = 3

_lib.rpq_set_option.argtypes = [c_void_p, ctypes.c_char_p, ctypes.c_double]
_lib.rpq_server_create.argtypes = [c_void_p, c_void_p, c_u64, c_u32, P(c_void_p)]
_lib.rpq_server_submit.argtypes = [c_void_p, P(rpq_request), P(c_u64)]
_lib.rpq_server_wait.argtypes = [c_void_p, c_u64, ctypes.c_double, P(rpq_reply)]
_lib.rpq_server_stats.argtypes = [c_void_p, P(c_u64), P(c_u64)]
_lib.rpq_server_cancel.argtypes = [c_void_p]
_lib.rpq_server_destroy.argtypes = [c_void_p]
_lib.rpq_server_destroy.restype = None
EXPORTED += ["rpq_set_option", "rpq_server_create", "rpq_server_submit", "rpq_server_wait", "rpq_server_stats",
             "rpq_server_cancel", "rpq_server_destroy"]


def rpq_set_option(ctx: Context, name: str, value: float):
    ctx.check(_lib.rpq_set_option(ctx.h, name.encode(), float(value)))


_lib.rpq_get_option.argtypes = [c_void_p, ctypes.c_char_p, P(ctypes.c_double)]
EXPORTED += ["rpq_get_option"]


def rpq_get_option(ctx: Context, name: str) -> float:
    v = ctypes.c_double()
    ctx.check(_lib.rpq_get_option(ctx.h, name.encode(), ctypes.byref(v)))
    return v.value


class rpq_server_counters(ctypes.Structure):
    _fields_ = [("launches", c_u64), ("admitted", c_u64), ("lane_requests", c_u64), ("lane_launches", c_u64),
                ("graph", c_u32), ("slots", c_u32)]


_lib.rpq_server_info.argtypes = [c_void_p, P(rpq_server_counters)]
EXPORTED += ["rpq_server_info"]


class Server:
    """rpq_server_*: continuous batching of mixed requests on one graph."""

    def __init__(self, ctx: Context, g: Graph, mem_budget_bytes: int = 0, max_batch: int = 4096):
        h = c_void_p()
        ctx.check(_lib.rpq_server_create(ctx.h, g.h, mem_budget_bytes, max_batch, ctypes.byref(h)))
        self.ctx, self.g, self.h = ctx, g, h
        self._keep = {}

    def submit_single(self, q: Query, source: int) -> int:
        return self._submit(rpq_request(RPQ_REQ_SINGLE, q.h, int(source), 0, None, None, 0), (q,))

    def submit_allpairs(self, q: Query) -> int:
        return self._submit(rpq_request(RPQ_REQ_ALLPAIRS, q.h, 0, 0, None, None, 0), (q,))

    def submit_crpq(self, n_vars: int, atoms, var_label=None) -> int:
        arr = (crpq_atom * len(atoms))(*[crpq_atom(a[0], a[2], a[1].h) for a in atoms])
        vl = None if var_label is None else np.ascontiguousarray(var_label, dtype=np.int32)
        req = rpq_request(RPQ_REQ_CRPQ, None, 0, n_vars, _ptr(vl), ctypes.cast(arr, c_void_p), len(atoms))
        return self._submit(req, tuple(a[1] for a in atoms))

    def _submit(self, req, keep) -> int:
        t = c_u64()
        rc = _lib.rpq_server_submit(self.h, ctypes.byref(req), ctypes.byref(t))
        if rc != 0:
            raise RPQError(rc, "submit refused")
        self._keep[t.value] = keep
        return t.value

    def wait(self, ticket: int, timeout_s: float = -1.0) -> dict:
        rep = rpq_reply()
        rc = _lib.rpq_server_wait(self.h, ticket, timeout_s, ctypes.byref(rep))
        if rc != 0:
            raise RPQError(rc, "wait failed")
        self._keep.pop(ticket, None)
        return rep.as_dict()

    def cancel(self):
        """Cancels every request not yet done (status RPQ_ERR_CANCELLED)."""
        _lib.rpq_server_cancel(self.h)

    def info(self) -> dict:
        """rpq_server_info: launches, admitted, lane_requests, lane_launches,
        graph (1 = serving launches replay a captured CUDA graph), slots."""
        c = rpq_server_counters()
        rc = _lib.rpq_server_info(self.h, ctypes.byref(c))
        if rc != 0:
            raise RPQError(rc, "server info failed")
        return {k: getattr(c, k) for k, _ in c._fields_}

    def stats(self):
        b, r = c_u64(), c_u64()
        _lib.rpq_server_stats(self.h, ctypes.byref(b), ctypes.byref(r))
        return b.value, r.value

    def close(self):
        if getattr(self, "h", None):
            _lib.rpq_server_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


# ---- streamed materialization ------------------------------------------------

class rpq_row_block(ctypes.Structure):
    _fields_ = [("n_sources", c_u32), ("sources", P(c_u32)), ("offsets", P(c_u64)), ("dst", P(c_u32)),
                ("n_rows", c_u64), ("query", c_u32)]


_lib.rpq_stream_open.argtypes = [c_void_p, c_void_p, c_void_p, c_u32, c_u32, c_u32, P(c_void_p)]
_lib.rpq_stream_open_multi.argtypes = [c_void_p, c_void_p, P(c_void_p), c_u32, c_u32, c_u32, c_u32, P(c_void_p)]
_lib.rpq_stream_next.argtypes = [c_void_p, P(rpq_row_block)]
_lib.rpq_stream_info.argtypes = [c_void_p, P(c_u64), P(c_u64), P(c_u64), P(rpq_stats)]
_lib.rpq_stream_close.argtypes = [c_void_p]
_lib.rpq_stream_close.restype = None
EXPORTED += ["rpq_stream_open", "rpq_stream_open_multi", "rpq_stream_next", "rpq_stream_info", "rpq_stream_close"]


class Stream:
    """rpq_stream_*: rows of rho from start vertices [begin, end), block by
    block, copied to the host while the device keeps exploring.  q is one
    Query or a sequence of them (rpq_stream_open_multi: the queries run one
    after another; ``block_query`` is the index of the last block's query)."""

    def __init__(self, ctx: Context, g: Graph, q, begin: int, end: int, flags: int = 0):
        h = c_void_p()
        if isinstance(q, Query):
            ctx.check(_lib.rpq_stream_open(ctx.h, g.h, q.h, begin, end, flags, ctypes.byref(h)))
        else:
            qs = list(q)
            arr = (c_void_p * max(1, len(qs)))(*[x.h for x in qs])
            ctx.check(_lib.rpq_stream_open_multi(ctx.h, g.h, arr, len(qs), begin, end, flags, ctypes.byref(h)))
        self.ctx, self.g, self.q, self.h = ctx, g, q, h
        self._blk = rpq_row_block()
        self.block_query = 0

    def next_block(self):
        """(sources, offsets, dst) as numpy views of the library's pinned slot
        (valid until the next call), or None at the end."""
        self.ctx.check(_lib.rpq_stream_next(self.h, ctypes.byref(self._blk)))
        b = self._blk
        if b.n_rows == 0:
            return None
        self.block_query = b.query
        src = np.ctypeslib.as_array(b.sources, shape=(b.n_sources,))
        off = np.ctypeslib.as_array(b.offsets, shape=(b.n_sources + 1,))
        dst = np.ctypeslib.as_array(b.dst, shape=(b.n_rows,))
        return src, off, dst

    def pairs(self) -> np.ndarray:
        """Every remaining row as an (n, 2) uint32 array (copied)."""
        out = []
        while (blk := self.next_block()) is not None:
            src, off, dst = blk
            out.append(np.stack([np.repeat(src, np.diff(off).astype(np.int64)), dst], axis=1).astype(np.uint32))
        return np.concatenate(out) if out else np.zeros((0, 2), dtype=np.uint32)

    def info(self):
        rows, s, x = c_u64(), c_u64(), c_u64()
        st = rpq_stats()
        _lib.rpq_stream_info(self.h, ctypes.byref(rows), ctypes.byref(s), ctypes.byref(x), ctypes.byref(st))
        return rows.value, s.value, x.value, st.as_dict()

    def close(self):
        if getattr(self, "h", None):
            _lib.rpq_stream_close(self.h)
            self.h = None

    def __del__(self):
        self.close()
