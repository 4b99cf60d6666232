"""Seeded synthetic inputs: labeled graphs, source samples and query strings.

This module holds no RPQ arithmetic; it only draws inputs.  Both the CUDA
path and the CPU oracle consume what it returns, so the two sides always see
identical inputs.  Random numbers come from numpy's PCG64 bit generator
through ``random_raw`` (a stable bit stream), never from distribution
methods whose algorithms may change between numpy versions.

Workloads (stand-ins for the paper's LDBC SNB / StackOverflow datasets,
which are not available; see Section 7.1 of the paper for those):

* ``er_graph``   -- directed Erdos-Renyi G(n, m): m distinct ordered pairs
  uniform over n x n (self-loops allowed), edge labels uniform.
* ``rmat_graph`` -- R-MAT with quadrant probabilities (a, b, c, d), a seeded
  Graph500-style vertex permutation, i.i.d. Zipf(s) edge labels.  Duplicate
  (src, dst, label) triples are left in; loading removes them.
"""

from __future__ import annotations

import numpy as np

BASE_SEED = 0x260220748

__all__ = [
    "BASE_SEED",
    "zipf_probs",
    "er_graph",
    "rmat_graph",
    "vertex_labels",
    "sample_sources",
    "random_regex",
    "random_graph",
]


def _raw(seed: int, n: int) -> np.ndarray:
    return np.random.Generator(np.random.PCG64(seed)).bit_generator.random_raw(n).astype(np.uint64)


class _Stream:
    """Chunked access to one PCG64 raw stream."""

    def __init__(self, seed: int):
        self.bg = np.random.PCG64(seed)

    def raw(self, n: int) -> np.ndarray:
        return self.bg.random_raw(n).astype(np.uint64)

    def unit(self, n: int) -> np.ndarray:
        """Uniform doubles in [0, 1) from the top 53 bits."""
        return (self.raw(n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))

    def below(self, n: int, k: int) -> np.ndarray:
        """Integers in [0, k) by the multiply-shift map of the top 32 bits."""
        hi = self.raw(n) >> np.uint64(32)
        return ((hi * np.uint64(k)) >> np.uint64(32)).astype(np.int64)


def zipf_probs(n_labels: int, s: float) -> np.ndarray:
    """P(label i) proportional to 1 / (i + 1)^s, i = 0 .. n_labels - 1."""
    w = 1.0 / np.arange(1, n_labels + 1, dtype=np.float64) ** s
    return w / w.sum()


def _zipf_labels(stream: _Stream, m: int, n_labels: int, s: float) -> np.ndarray:
    cdf = np.cumsum(zipf_probs(n_labels, s))
    cdf[-1] = 1.0
    lab = np.searchsorted(cdf, stream.unit(m), side="right")
    return np.minimum(lab, n_labels - 1).astype(np.uint16)


def er_graph(n: int, m: int, n_labels: int, seed: int):
    """m distinct ordered pairs uniform over n x n, labels uniform."""
    if m > n * n:
        raise ValueError("m exceeds n^2")
    st = _Stream(seed)
    chosen = np.empty(0, dtype=np.int64)
    while len(chosen) < m:
        cand = st.below(2 * (m - len(chosen)) + 16, n * n)
        merged = np.concatenate([chosen, cand])
        _, first = np.unique(merged, return_index=True)
        first.sort()
        chosen = merged[first][:m]
    src = (chosen // n).astype(np.uint32)
    dst = (chosen % n).astype(np.uint32)
    lab = st.below(m, n_labels).astype(np.uint16)
    return src, dst, lab


def rmat_graph(scale: int, n_edges: int, n_labels: int, zipf_s: float, seed: int,
               probs=(0.57, 0.19, 0.19, 0.05), permute: bool = True, chunk: int = 1 << 22):
    """R-MAT edges (src, dst, label) over 2^scale vertices."""
    a, b, c, _ = probs
    t1 = np.uint64(int(a * 2**32))
    t2 = np.uint64(int((a + b) * 2**32))
    t3 = np.uint64(int((a + b + c) * 2**32))
    st = _Stream(seed)
    src = np.empty(n_edges, dtype=np.uint32)
    dst = np.empty(n_edges, dtype=np.uint32)
    words = (scale + 1) // 2
    lo_mask = np.uint64(0xFFFFFFFF)
    for c0 in range(0, n_edges, chunk):
        k = min(chunk, n_edges - c0)
        s = np.zeros(k, dtype=np.uint32)
        d = np.zeros(k, dtype=np.uint32)
        level = 0
        for _ in range(words):
            r = st.raw(k)
            for u in (r >> np.uint64(32), r & lo_mask):
                if level == scale:
                    break
                bit = np.uint32(1 << level)
                # quadrants: u < a -> (0,0); < a+b -> (0,1); < a+b+c -> (1,0); else (1,1)
                sb = u >= t2
                db = ((u >= t1) & (u < t2)) | (u >= t3)
                s |= sb.astype(np.uint32) * bit
                d |= db.astype(np.uint32) * bit
                level += 1
        src[c0:c0 + k] = s
        dst[c0:c0 + k] = d
    if permute:
        perm = np.argsort(_raw(seed ^ 0x5EED_0001, 1 << scale), kind="stable").astype(np.uint32)
        src = perm[src]
        dst = perm[dst]
    lab = _zipf_labels(_Stream(seed ^ 0x5EED_0002), n_edges, n_labels, zipf_s)
    return src, dst, lab


def vertex_labels(n: int, n_vlabels: int, seed: int) -> np.ndarray:
    return _Stream(seed ^ 0x5EED_0003).below(n, n_vlabels).astype(np.uint8)


def sample_sources(n_vertices: int, src: np.ndarray, seed: int, n_strat: int = 256, n_hubs: int = 128,
                   n_uniform: int = 128) -> np.ndarray:
    """Seeded source sample: ``n_strat`` stratified by out-degree decile (over
    vertices with out-degree > 0), the ``n_hubs`` highest out-degree vertices
    and ``n_uniform`` uniform vertices.  Sorted, distinct."""
    deg = np.bincount(np.asarray(src, dtype=np.int64), minlength=n_vertices)
    st = _Stream(seed ^ 0x5EED_0004)
    picked = []
    nz = np.nonzero(deg)[0]
    if len(nz):
        order = nz[np.argsort(deg[nz], kind="stable")]
        deciles = np.array_split(order, 10)
        per = max(1, n_strat // 10)
        for dec in deciles:
            if len(dec):
                picked.append(dec[st.below(per, len(dec))])
    hubs = np.argsort(-deg, kind="stable")[:n_hubs]
    picked.append(hubs)
    picked.append(st.below(n_uniform, n_vertices))
    return np.unique(np.concatenate(picked)).astype(np.uint32)


def random_graph(n: int, m: int, n_labels: int, seed: int):
    """Small multigraph for brute-force checks: m uniform (src, dst, label)
    draws (duplicates and self-loops possible)."""
    st = _Stream(seed)
    return (st.below(m, n).astype(np.uint32), st.below(m, n).astype(np.uint32),
            st.below(m, n_labels).astype(np.uint16))


def random_regex(seed: int, n_labels: int, max_symbols: int = 5, p_star: float = 0.35,
                 p_alt: float = 0.25) -> str:
    """A random regex over single-letter labels: 1..max_symbols symbols, each
    optionally starred / plussed / optional, adjacent pairs sometimes grouped
    as an alternation, an occasional outer group with a postfix."""
    st = _Stream(seed)
    u = st.unit(64)
    idx = [0]

    def nxt():
        x = u[idx[0] % 64]
        idx[0] += 1
        return x

    k = 1 + int(nxt() * max_symbols)
    parts = []
    i = 0
    while i < k:
        sym = chr(ord("a") + int(nxt() * n_labels))
        if i + 1 < k and nxt() < p_alt:
            sym2 = chr(ord("a") + int(nxt() * n_labels))
            tok = f"({sym}|{sym2})"
            i += 2
        else:
            tok = sym
            i += 1
        r = nxt()
        if r < p_star:
            tok += "*"
        elif r < p_star + 0.1:
            tok += "+"
        elif r < p_star + 0.18:
            tok += "?"
        parts.append(tok)
    text = ".".join(parts)
    r = nxt()
    if len(parts) > 1 and r < 0.15:
        text = f"({text})*"
    elif len(parts) > 1 and r < 0.22:
        text = f"({text})+"
    return text


def _draw_regex(st: _Stream, cdf: np.ndarray, n_ranks: int, first_rank: int) -> str:
    """One regex of the single-source mix: 1..6 symbols, each a label of rank
    first_rank + (a draw from cdf); stars on k in {0, 1, 2} distinct symbols;
    with probability 1/4 two adjacent symbols become an alternation."""
    k = 1 + int(st.below(1, 6)[0])
    syms = [chr(ord("a") + first_rank + min(int(np.searchsorted(cdf, st.unit(1)[0], side="right")), n_ranks - 1))
            for _ in range(k)]
    n_star = min(k, int(st.below(1, 3)[0]))
    starred = set()
    while len(starred) < n_star:
        starred.add(int(st.below(1, k)[0]))
    parts = [s + ("*" if i in starred else "") for i, s in enumerate(syms)]
    if k >= 2 and st.unit(1)[0] < 0.25:
        i = int(st.below(1, k - 1)[0])
        a, b = syms[i], syms[i + 1]
        star = "*" if (i in starred or i + 1 in starred) else ""
        parts = parts[:i] + [f"({a}|{b}){star}"] + parts[i + 2:]
    return ".".join(parts)


def _degree_sources(st: _Stream, n: int, src: np.ndarray, n_vertices: int) -> np.ndarray:
    deg = np.bincount(np.asarray(src, dtype=np.int64), minlength=n_vertices).astype(np.float64)
    cum = np.cumsum(deg)
    u = st.unit(n) * cum[-1]
    return np.minimum(np.searchsorted(cum, u, side="right"), n_vertices - 1).astype(np.uint32)


def batch_queries(n_queries: int, n_labels: int, zipf_s: float, src: np.ndarray, n_vertices: int, seed: int):
    """Single-source query mix: each regex has 1..6 symbols, each a label drawn
    Zipf(zipf_s); Kleene stars on k in {0, 1, 2} (uniform) distinct symbols; with
    probability 1/4 two adjacent symbols are grouped as an alternation.  Start
    vertices are drawn with probability proportional to out-degree (with
    replacement).  Returns (list of regex strings, uint32 sources)."""
    st = _Stream(seed)
    cdf = np.cumsum(zipf_probs(n_labels, zipf_s))
    cdf[-1] = 1.0
    regexes = [_draw_regex(st, cdf, n_labels, 0) for _ in range(n_queries)]
    return regexes, _degree_sources(st, n_queries, src, n_vertices)


def serve_stream(rate: float, seconds: float, n_labels: int, zipf_s: float, src: np.ndarray, n_vertices: int,
                 seed: int, mix=(0.80, 0.15, 0.05), tail_rank: int = 8):
    """Mixed request stream with Poisson arrivals (mean `rate` per second over
    `seconds`).  Each request is, with the probabilities of `mix`:
    1 single-source -- a regex of the batch_queries mix from a start vertex
      drawn proportional to out-degree;
    2 all-pairs -- a regex of the same shape whose labels come from the Zipf
      tail (ranks tail_rank .. n_labels - 1, Zipf(zipf_s) renormalized there);
    3 CRPQ -- the triangle x -l1-> y, x -l2.l3*-> z, y -l4*-> z with l1..l4
      drawn from the same tail.
    Returns (t: arrival seconds ascending, kind: uint8, spec: list) where spec
    is (regex, source), regex, or (l1, l2, l3, l4) as label letters."""
    st = _Stream(seed)
    gaps = -np.log1p(-st.unit(int(rate * seconds * 1.2) + 64)) / rate
    t = np.cumsum(gaps)
    t = t[t < seconds]
    m = len(t)
    u = st.unit(m)
    kind = np.where(u < mix[0], 1, np.where(u < mix[0] + mix[1], 2, 3)).astype(np.uint8)
    head = np.cumsum(zipf_probs(n_labels, zipf_s))
    head[-1] = 1.0
    n_tail = n_labels - tail_rank
    tw = zipf_probs(n_labels, zipf_s)[tail_rank:]
    tail = np.cumsum(tw / tw.sum())
    tail[-1] = 1.0
    srcs = _degree_sources(st, m, src, n_vertices)

    def tail_letter():
        return chr(ord("a") + tail_rank + min(int(np.searchsorted(tail, st.unit(1)[0], side="right")), n_tail - 1))

    spec = []
    for i in range(m):
        if kind[i] == 1:
            spec.append((_draw_regex(st, head, n_labels, 0), int(srcs[i])))
        elif kind[i] == 2:
            spec.append(_draw_regex(st, tail, n_tail, tail_rank))
        else:
            spec.append(tuple(tail_letter() for _ in range(4)))
    return t, kind, spec
