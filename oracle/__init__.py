"""CPU oracle for RPQ / CRPQ evaluation.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and
``bench.py``'s cpu_baseline / reference legs may import this package.  It
shares no code with the CUDA path and never imports it.

* ``rpq_oracle.cpp`` -- product-graph BFS over a Thompson epsilon-NFA
  (Definition 1, Section 2.2 automata-based approach), CRPQ by nested loops
  (Definition 2), and the product-edge work counter W over the minimal DFA.
* ``algebra.py`` -- boolean-matrix algebra (Section 2.2 algebra-based
  approach) for small graphs: an independent second algorithm.
* ``splitmix64`` / ``pair_hash`` -- the order-independent result digest.

Parity status: all functions are pinned by tests/test_oracle_pins.py.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rpq_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liborc.so")
_lib = None

GOLDEN_GAMMA = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1


def build(force: bool = False) -> str:
    """Compiles the oracle shared library with g++ (OpenMP over sources)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["g++", "-O2", "-std=c++17", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC]
        )
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    c = ctypes
    lib.orc_last_error.restype = c.c_char_p
    lib.orc_graph_new.argtypes = [c.c_uint32, c.c_uint32, c.c_uint64, c.c_void_p, c.c_void_p, c.c_void_p,
                                  c.c_void_p, c.POINTER(c.c_void_p)]
    lib.orc_graph_free.argtypes = [c.c_void_p]
    lib.orc_graph_edges.argtypes = [c.c_void_p]
    lib.orc_graph_edges.restype = c.c_uint64
    lib.orc_dfa.argtypes = [c.c_char_p, c.c_void_p, c.c_uint32, c.c_uint32, c.c_int, c.POINTER(c.c_int),
                            c.c_void_p, c.c_void_p]
    lib.orc_rpq.argtypes = [c.c_void_p, c.c_char_p, c.c_void_p, c.c_uint32, c.c_void_p, c.c_uint64, c.c_int,
                            c.POINTER(c.c_void_p)]
    lib.orc_crpq.argtypes = [c.c_void_p, c.c_uint32, c.c_void_p, c.c_uint32, c.c_void_p, c.c_void_p, c.c_void_p,
                             c.c_void_p, c.c_uint32, c.c_void_p, c.c_uint64, c.c_int, c.POINTER(c.c_void_p)]
    lib.orc_result_rows.argtypes = [c.c_void_p]
    lib.orc_result_rows.restype = c.c_uint64
    lib.orc_result_arity.argtypes = [c.c_void_p]
    lib.orc_result_arity.restype = c.c_uint32
    lib.orc_result_copy.argtypes = [c.c_void_p, c.c_void_p]
    lib.orc_result_work.argtypes = [c.c_void_p, c.POINTER(c.c_uint64), c.POINTER(c.c_uint64),
                                    c.POINTER(c.c_uint64), c.POINTER(c.c_int)]
    lib.orc_result_free.argtypes = [c.c_void_p]
    _lib = lib
    return lib


class OracleError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"oracle error {code}: {msg}")
        self.code = code


def _check(rc: int):
    if rc != 0:
        raise OracleError(rc, _load().orc_last_error().decode())


def _names_arg(names):
    if names is None:
        return None, 0, None
    arr = (ctypes.c_char_p * len(names))(*[n.encode() for n in names])
    return ctypes.cast(arr, ctypes.c_void_p), len(names), arr


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class Graph:
    """Deduplicated labeled graph held by the oracle."""

    def __init__(self, n_vertices, n_labels, src, dst, label, vertex_label=None):
        lib = _load()
        self._src = np.ascontiguousarray(src, dtype=np.uint32)
        self._dst = np.ascontiguousarray(dst, dtype=np.uint32)
        self._lab = np.ascontiguousarray(label, dtype=np.uint16)
        self._vl = None if vertex_label is None else np.ascontiguousarray(vertex_label, dtype=np.uint8)
        h = ctypes.c_void_p()
        _check(lib.orc_graph_new(n_vertices, n_labels, len(self._src), _ptr(self._src), _ptr(self._dst),
                                 _ptr(self._lab), _ptr(self._vl), ctypes.byref(h)))
        self.h = h
        self.n_vertices = n_vertices
        self.n_labels = n_labels

    @property
    def n_edges(self) -> int:
        return int(_load().orc_graph_edges(self.h))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_graph_free(self.h)
            self.h = None


class Result:
    def __init__(self, rows: np.ndarray, W: int, N: int, mismatch: int, threads: int):
        self.rows = rows
        self.W = W
        self.N = N
        self.automaton_mismatch = mismatch
        self.threads = threads


def _take(h) -> Result:
    lib = _load()
    n = lib.orc_result_rows(h)
    k = lib.orc_result_arity(h)
    rows = np.empty((n, k), dtype=np.uint32)
    if n:
        lib.orc_result_copy(h, rows.ctypes.data_as(ctypes.c_void_p))
    W, N, mm, th = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_int()
    lib.orc_result_work(h, ctypes.byref(W), ctypes.byref(N), ctypes.byref(mm), ctypes.byref(th))
    lib.orc_result_free(h)
    return Result(rows, W.value, N.value, mm.value, th.value)


def rpq(graph: Graph, regex: str, sources=None, names=None, threads: int = 0) -> Result:
    """Definition 1: distinct (src, dst) pairs, sorted, from each start vertex
    (all vertices when ``sources`` is None)."""
    lib = _load()
    nptr, nn, keep = _names_arg(names)
    srcs = None if sources is None else np.ascontiguousarray(sources, dtype=np.uint32)
    h = ctypes.c_void_p()
    _check(lib.orc_rpq(graph.h, regex.encode(), nptr, nn, _ptr(srcs), 0 if srcs is None else len(srcs),
                       threads, ctypes.byref(h)))
    del keep
    return _take(h)


def crpq(graph: Graph, n_vars: int, atoms, var_label=None, restrict0=None, names=None, threads: int = 0) -> Result:
    """Definition 2.  ``atoms`` is a list of (x, regex, y) with variable
    indices x, y.  Rows are distinct tuples in variable order, sorted."""
    lib = _load()
    nptr, nn, keep = _names_arg(names)
    ax = np.array([a[0] for a in atoms], dtype=np.uint32)
    ay = np.array([a[2] for a in atoms], dtype=np.uint32)
    res = (ctypes.c_char_p * len(atoms))(*[a[1].encode() for a in atoms])
    vl = None if var_label is None else np.ascontiguousarray(var_label, dtype=np.int32)
    r0 = None if restrict0 is None else np.ascontiguousarray(restrict0, dtype=np.uint32)
    h = ctypes.c_void_p()
    _check(lib.orc_crpq(graph.h, n_vars, _ptr(vl), len(atoms), _ptr(ax), _ptr(ay),
                        ctypes.cast(res, ctypes.c_void_p), nptr, nn, _ptr(r0), 0 if r0 is None else len(r0),
                        threads, ctypes.byref(h)))
    del keep
    return _take(h)


def dfa(regex: str, n_labels: int, names=None, max_states: int = 256):
    """The oracle's minimal DFA: (n_states, final[n], next[n, n_labels])."""
    lib = _load()
    nptr, nn, keep = _names_arg(names)
    n = ctypes.c_int()
    fin = np.zeros(max_states, dtype=np.uint8)
    nxt = np.full(max_states * n_labels, -1, dtype=np.int32)
    _check(lib.orc_dfa(regex.encode(), nptr, nn, n_labels, max_states, ctypes.byref(n), _ptr(fin), _ptr(nxt)))
    del keep
    k = n.value
    return k, fin[:k].astype(bool), nxt[: k * n_labels].reshape(k, n_labels)


def splitmix64(x):
    """SplitMix64 output for state ``x`` (Steele, Lea, Flood 2014): the state
    is advanced by the golden gamma and the result is put through the
    variant-13 finalizer.  Works on Python ints and uint64 numpy arrays."""
    if isinstance(x, np.ndarray):
        with np.errstate(over="ignore"):
            z = x.astype(np.uint64) + np.uint64(GOLDEN_GAMMA)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            return z ^ (z >> np.uint64(31))
    z = (x + GOLDEN_GAMMA) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def row_digest(rows: np.ndarray):
    """Order-independent digest of a set of rows t[0..k-1]:
    (count, sum mod 2^64, xor) of h(row), where h = s(t0) for k = 1 and
    h = s(t0 << 32 | t1) folded with s(h ^ t_i) for each further column
    (s = splitmix64)."""
    rows = np.asarray(rows, dtype=np.uint64)
    if rows.ndim == 1:
        rows = rows.reshape(-1, 1)
    if len(rows) == 0:
        return 0, 0, 0
    k = rows.shape[1]
    if k == 1:
        h = splitmix64(rows[:, 0])
    else:
        h = splitmix64((rows[:, 0] << np.uint64(32)) | rows[:, 1])
        for i in range(2, k):
            h = splitmix64(h ^ rows[:, i])
    with np.errstate(over="ignore"):
        s = int(np.add.reduce(h, dtype=np.uint64))
    x = int(np.bitwise_xor.reduce(h))
    return len(rows), s, x


def pair_digest(rows: np.ndarray):
    """``row_digest`` of (src, dst) rows."""
    return row_digest(np.asarray(rows).reshape(-1, 2))
