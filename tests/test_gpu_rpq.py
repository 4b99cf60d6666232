"""GPU parity of RPQ evaluation against the CPU oracle, through the C ABI.

Bit-exact comparison of the sorted distinct (src, dst) rows, of the row
digest (count, sum, xor of splitmix64) and of the product-edge work counter W,
on the paper's worked example, the small ER configuration in full, random
graphs x random regexes in both expansion directions and both lane widths,
edge cases, and sampled sources of the large R-MAT configuration in the
launch configuration the benchmark uses."""

import os

import numpy as np
import pytest

import oracle
from paper_2602_20748_gb300 import synth
from conftest import load_graph_fixture, load_rows

pytestmark = pytest.mark.gpu

rpq = pytest.importorskip("paper_2602_20748_gb300.rpq")

MODES = {
    "auto": 0,
    "push": rpq.RPQ_FORCE_PUSH,
    "pull": rpq.RPQ_FORCE_PULL,
}


@pytest.fixture(scope="module")
def ctx():
    return rpq.Context(device=0)


def gpu_rows(ctx, g, regex, sources=None, mode=0, names=None):
    q = rpq.compile_rpq(ctx, regex, names)
    r = rpq.run_rpq(ctx, g, q, sources, flags=rpq.RPQ_MATERIALIZE | mode)
    rows = rpq.fetch_pairs(r)
    info = rpq.result_info(r)
    st = rpq.result_stats(r)
    return rows, info, st


def check(ctx, g, og, regex, sources=None, mode=0, names=None, want=None):
    if want is None:
        want = oracle.rpq(og, regex, sources=sources, names=names)
    rows, info, st = gpu_rows(ctx, g, regex, sources, mode, names)
    assert rows.shape == want.rows.shape, (regex, len(rows), len(want.rows))
    assert np.array_equal(rows, want.rows), regex
    cnt, s, x = oracle.pair_digest(want.rows)
    assert info[0] == cnt and info[2] == s and info[3] == x
    assert st["product_edges"] == want.W, (regex, st["product_edges"], want.W)
    assert st["product_vertices"] == want.N
    return rows, st


def test_fig1_q1(ctx):
    n, L, src, dst, lab, _ = load_graph_fixture("fig1_graph.txt")
    g = rpq.load_graph(ctx, n, L, src, dst, lab)
    for name, mode in MODES.items():
        rows, _, _ = gpu_rows(ctx, g, "abc*", mode=mode)
        assert rows.tolist() == load_rows("fig1_q1_abcstar.txt").tolist(), name
    rows, _, _ = gpu_rows(ctx, g, "abc*", sources=[0])
    assert len(rows) == 9
    assert g.info() == (14, 3, 19)


@pytest.fixture(scope="module")
def er1000(ctx):
    src, dst, lab = synth.er_graph(1000, 5000, 4, seed=synth.BASE_SEED + 0)
    return rpq.load_graph(ctx, 1000, 4, src, dst, lab), oracle.Graph(1000, 4, src, dst, lab)


@pytest.mark.parametrize("mode", list(MODES))
def test_er_config_abcstar_full(ctx, er1000, mode):
    """All-pairs a.b.c* on the seeded ER graph (1,000 vertices, 5,000 edges,
    4 uniform labels), in full."""
    g, og = er1000
    check(ctx, g, og, "a.b.c*", mode=MODES[mode])


@pytest.mark.parametrize("regex", ["a*", "(a|b)+.c", "a.b*.c", "(a.b)*", "a?b*", "abcd", "(a|b|c)*", "d",
                                   "c.c.c", "(a.b|c.d)+", "a*b*"])
def test_er_regex_zoo(ctx, er1000, regex):
    g, og = er1000
    check(ctx, g, og, regex)


def test_er_count_only_matches_materialized(ctx, er1000):
    g, og = er1000
    q = rpq.compile_rpq(ctx, "(a|b)+.c")
    r1 = rpq.run_rpq(ctx, g, q, flags=rpq.RPQ_MATERIALIZE)
    r2 = rpq.run_rpq(ctx, g, q, flags=rpq.RPQ_COUNT_ONLY)
    assert rpq.result_info(r1) == rpq.result_info(r2)
    with pytest.raises(rpq.RPQError):
        rpq.fetch_pairs(r2)


def test_er_fetch_slices(ctx, er1000):
    g, og = er1000
    q = rpq.compile_rpq(ctx, "a*")
    r = rpq.run_rpq(ctx, g, q)
    full = rpq.fetch_pairs(r)
    parts = [rpq.fetch_pairs(r, off, 777) for off in range(0, len(full), 777)]
    assert np.array_equal(np.concatenate(parts), full)
    assert len(rpq.fetch_pairs(r, len(full) + 5, 10)) == 0


@pytest.mark.parametrize("case", range(40))
def test_random_graphs_both_directions(ctx, case):
    n = 37 + 53 * (case % 7)
    L = 2 + case % 4
    src, dst, lab = synth.random_graph(n, n * (2 + case % 5), L, seed=7000 + case)
    regex = synth.random_regex(8000 + case, L, max_symbols=5)
    g = rpq.load_graph(ctx, n, L, src, dst, lab)
    og = oracle.Graph(n, L, src, dst, lab)
    want = oracle.rpq(og, regex)
    for mode in MODES.values():
        check(ctx, g, og, regex, mode=mode, want=want)
    # a short source list (one 64-lane group) with duplicates, unsorted
    sources = np.array([n - 1, 3, 3, 0, n // 2], dtype=np.uint32)
    want = oracle.rpq(og, regex, sources=sources)
    for mode in MODES.values():
        check(ctx, g, og, regex, sources=sources, mode=mode, want=want)


def test_many_groups_and_batches(ctx):
    """More lane groups than one launch holds: several launches, results
    concatenated in source order."""
    n, L = 3000, 3
    src, dst, lab = synth.rmat_graph(12, 4 * n, L, 1.2, seed=99)
    src %= n
    dst %= n
    old = os.environ.get("RPQ_MAX_GROUPS")
    os.environ["RPQ_MAX_GROUPS"] = "2"
    try:
        c2 = rpq.Context(device=0)
    finally:
        if old is None:
            del os.environ["RPQ_MAX_GROUPS"]
        else:
            os.environ["RPQ_MAX_GROUPS"] = old
    g = rpq.load_graph(c2, n, L, src, dst, lab)
    og = oracle.Graph(n, L, src, dst, lab)
    for regex in ("a*", "a.b*.c", "(a|b)+"):
        rows, st = check(c2, g, og, regex)
        assert st["lane_groups"] == (n + 255) // 256


def test_edge_cases(ctx):
    # no edges at all: only the empty word can match
    g = rpq.load_graph(ctx, 5, 2, [], [], [])
    rows, info, _ = gpu_rows(ctx, g, "a*")
    assert rows.tolist() == [[v, v] for v in range(5)]
    rows, info, _ = gpu_rows(ctx, g, "a")
    assert len(rows) == 0
    # duplicates, self-loops, parallel edges with different labels, a label
    # the graph does not have
    src = [0, 0, 0, 1, 1, 2, 3]
    dst = [1, 1, 1, 1, 2, 0, 3]
    lab = [0, 0, 1, 0, 1, 0, 1]
    g = rpq.load_graph(ctx, 6, 2, src, dst, lab)
    assert g.info() == (6, 2, 6)
    og = oracle.Graph(6, 2, src, dst, lab)
    for regex in ("a*", "a+", "b*", "(a|b)*", "a.b", "z", "a|z", "z*", "a.z*.b"):
        for mode in MODES.values():
            check(ctx, g, og, regex, mode=mode)
    # single vertex
    g1 = rpq.load_graph(ctx, 1, 1, [0], [0], [0])
    og1 = oracle.Graph(1, 1, [0], [0], [0])
    for regex in ("a", "a*", "a.a.a"):
        check(ctx, g1, og1, regex)


def test_heavy_vertices(ctx):
    """Hubs far above the high-degree threshold in both directions: vertex 0
    has in-degree 3,000 (label a), vertex 1 out-degree 2,500 (label b)."""
    n = 4000
    rs, rd, rl = synth.random_graph(n, 6000, 3, seed=77)
    src = np.concatenate([np.arange(1, 3001), np.ones(2500), rs]).astype(np.uint32)
    dst = np.concatenate([np.zeros(3000), np.arange(1500, 4000), rd]).astype(np.uint32)
    lab = np.concatenate([np.zeros(3000), np.ones(2500), rl]).astype(np.uint16)
    g = rpq.load_graph(ctx, n, 3, src, dst, lab)
    og = oracle.Graph(n, 3, src, dst, lab)
    sample = np.arange(0, n, 7, dtype=np.uint32)
    for regex in ("a.b", "(a|b)*", "a*.b.c*", "(a.b)+"):
        want = oracle.rpq(og, regex, sources=sample)
        for mode in MODES.values():
            check(ctx, g, og, regex, sources=sample, mode=mode, want=want)
        wrev = rpq.fetch_pairs(rpq.run_rpq(ctx, g, rpq.compile_rpq(ctx, regex), np.array([0, 1, 2000], np.uint32),
                                           flags=rpq.RPQ_MATERIALIZE | rpq.RPQ_REVERSE | rpq.RPQ_FORCE_PULL))
        full = oracle.rpq(og, regex).rows
        want_rev = sorted((int(d), int(s)) for s, d in full.tolist() if d in (0, 1, 2000))
        assert [tuple(r) for r in wrev.tolist()] == want_rev


def test_invalid_arguments(ctx):
    with pytest.raises(rpq.RPQError) as e:
        rpq.load_graph(ctx, 4, 1, [0], [9], [0])
    assert e.value.code == rpq.RPQ_ERR_INVALID_ARG
    with pytest.raises(rpq.RPQError) as e:
        rpq.load_graph(ctx, 4, 1, [0], [1], [3])
    assert e.value.code == rpq.RPQ_ERR_INVALID_ARG
    g = rpq.load_graph(ctx, 4, 1, [0], [1], [0])
    q = rpq.compile_rpq(ctx, "a")
    with pytest.raises(rpq.RPQError) as e:
        rpq.run_rpq(ctx, g, q, [4])
    assert e.value.code == rpq.RPQ_ERR_INVALID_ARG
    with pytest.raises(rpq.RPQError) as e:
        rpq.run_rpq(ctx, g, q, flags=rpq.RPQ_MATERIALIZE | rpq.RPQ_COUNT_ONLY)
    assert e.value.code == rpq.RPQ_ERR_INVALID_ARG
    with pytest.raises(rpq.RPQError) as e:
        rpq.run_rpq_range(ctx, g, q, 3, 5)
    assert e.value.code == rpq.RPQ_ERR_INVALID_ARG


def test_range_batches_concatenate(ctx, er1000):
    g, og = er1000
    q = rpq.compile_rpq(ctx, "a.b*.c")
    full = rpq.fetch_pairs(rpq.run_rpq(ctx, g, q))
    parts = [rpq.fetch_pairs(rpq.run_rpq_range(ctx, g, q, b, min(1000, b + 300))) for b in range(0, 1000, 300)]
    assert np.array_equal(np.concatenate(parts), full)


def test_budget_exceeded_is_reported(ctx):
    small = rpq.Context(device=0, mem_budget_bytes=1 << 20)
    src, dst, lab = synth.er_graph(20000, 100000, 2, seed=5)
    with pytest.raises(rpq.RPQError) as e:
        rpq.load_graph(small, 20000, 2, src, dst, lab)
    assert e.value.code == rpq.RPQ_ERR_OUT_OF_BUDGET


# ---------------------------------------------------------------------------
# Large R-MAT configuration: 2^20 vertices, 2^24 generated edges, 8 labels
# Zipf(1.2), in the benchmark's launch configuration; sampled sources.
# ---------------------------------------------------------------------------

RMAT20 = dict(scale=20, n_edges=1 << 24, n_labels=8, zipf_s=1.2, seed=synth.BASE_SEED + 1)
RMAT20_QUERIES = ["a*", "(a|b)+·c", "a·b*·c", "(a·b)*"]


@pytest.fixture(scope="module")
def rmat20(ctx):
    src, dst, lab = synth.rmat_graph(**RMAT20)
    n = 1 << 20
    return (rpq.load_graph(ctx, n, 8, src, dst, lab), oracle.Graph(n, 8, src, dst, lab), src)


def test_rmat20_bench_batch_sampled(ctx, rmat20):
    """The benchmark's step: a batch of 4,096 consecutive start vertices per
    query, materialized.  Check sampled sources of the batch row by row
    against the oracle, and the whole batch's digest against count-only."""
    g, og, src = rmat20
    begin, end = 4096, 8192
    rng = np.random.Generator(np.random.PCG64(17))
    sample = np.unique(np.concatenate([rng.integers(begin, end, 40),
                                       # the highest-degree vertices of the batch
                                       begin + np.argsort(-np.bincount(src, minlength=1 << 20)[begin:end])[:8]]))
    for regex in RMAT20_QUERIES:
        q = rpq.compile_rpq(ctx, regex)
        r = rpq.run_rpq_range(ctx, g, q, begin, end)
        rows = rpq.fetch_pairs(r)
        want = oracle.rpq(og, regex, sources=sample)
        got = rows[np.isin(rows[:, 0], sample)]
        assert np.array_equal(got, want.rows), regex
        rc = rpq.run_rpq_range(ctx, g, q, begin, end, flags=rpq.RPQ_COUNT_ONLY)
        assert rpq.result_info(rc) == rpq.result_info(r)
        # rows are sorted and distinct
        keys = rows[:, 0].astype(np.uint64) << np.uint64(32) | rows[:, 1]
        assert np.all(keys[1:] > keys[:-1])


@pytest.mark.parametrize("regex", RMAT20_QUERIES)
def test_rmat20_sampled_sources_work_counter(ctx, rmat20, regex):
    """Stratified + hub + uniform sample of start vertices: rows, digest and
    the work counter W bit-exact against the oracle."""
    g, og, src = rmat20
    sample = synth.sample_sources(1 << 20, src, seed=3, n_strat=60, n_hubs=12, n_uniform=20)
    want = oracle.rpq(og, regex, sources=sample)
    for mode in MODES.values():
        check(ctx, g, og, regex, sources=sample, mode=mode, want=want)


def _ctx_with_env(**env):
    old = {k: os.environ.get(k) for k in env}
    os.environ.update({k: str(v) for k, v in env.items()})
    try:
        return rpq.Context(device=0)
    finally:
        for k, v in old.items():
            if v is None:
                del os.environ[k]
            else:
                os.environ[k] = v


def _hub_graph():
    # ten hubs with 2,500 out-edges (three 1,024-edge chunks each) plus noise
    n = 6000
    rs, rd, rl = synth.random_graph(n, 12000, 2, seed=91)
    hub_src = np.repeat(np.arange(10, dtype=np.uint32), 2500)
    hub_dst = synth.random_graph(n, 25000, 1, seed=92)[1]
    src = np.concatenate([hub_src, rs]).astype(np.uint32)
    dst = np.concatenate([hub_dst, rd]).astype(np.uint32)
    lab = np.concatenate([np.zeros(25000, np.uint16), rl]).astype(np.uint16)
    return n, src, dst, lab


def test_spill_capacity_overflow_falls_back_in_place():
    """Top-down rows longer than 1,024 edges are queued as chunks; when the
    per-level chunk capacity runs out, the remaining rows are processed in
    place (capacity forced down to 3 chunks here)."""
    c3 = _ctx_with_env(RPQ_SPILL_CAP=3)
    n, src, dst, lab = _hub_graph()
    g = rpq.load_graph(c3, n, 2, src, dst, lab)
    og = oracle.Graph(n, 2, src, dst, lab)
    sources = np.concatenate([np.arange(10), np.arange(100, 400)]).astype(np.uint32)
    for regex in ("a.b*", "(a|b)+"):
        want = oracle.rpq(og, regex, sources=sources)
        for mode in (0, rpq.RPQ_FORCE_PUSH):
            check(c3, g, og, regex, sources=sources, mode=mode, want=want)


@pytest.mark.parametrize("regex", ["a*", "a.b*", "(a|b)+", "b?"])
@pytest.mark.parametrize("flags", ["count", "rows"])
def test_edgeless_start_vertices_skipped(ctx, regex, flags):
    """Long source lists drop start vertices without an edge on the start
    state's labels; their (s, s) rows (when the start state accepts) are still
    counted and digested, and rows, digests, W and N stay exact."""
    n = 9000
    src, dst, lab = synth.random_graph(n, 3000, 3, seed=77)  # most vertices have no out-edge
    g = rpq.load_graph(ctx, n, 3, src, dst, lab)
    og = oracle.Graph(n, 3, src, dst, lab)
    want = oracle.rpq(og, regex)
    q = rpq.compile_rpq(ctx, regex)
    f = rpq.RPQ_COUNT_ONLY if flags == "count" else rpq.RPQ_MATERIALIZE
    r = rpq.run_rpq(ctx, g, q, None, flags=f)
    cnt, s, x = oracle.pair_digest(want.rows)
    assert rpq.result_info(r) == (cnt, 2, s, x)
    st = rpq.result_stats(r)
    assert st["product_edges"] == want.W and st["product_vertices"] == want.N
    if flags == "rows":
        assert np.array_equal(rpq.fetch_pairs(r), want.rows)


def test_static_chunk_order_matches_oracle():
    """pull_dynamic = 0: bottom-up levels take their 32-vertex chunks
    round-robin instead of from the cursor; every level bottom-up, hubs in
    both directions -- the rows and the work counter equal the oracle's."""
    c = rpq.Context(device=0)
    rpq.rpq_set_option(c, "pull_dynamic", 0)
    n = 4000
    rs, rd, rl = synth.random_graph(n, 6000, 3, seed=79)
    src = np.concatenate([np.arange(1, 3001), np.ones(2500), rs]).astype(np.uint32)
    dst = np.concatenate([np.zeros(3000), np.arange(1500, 4000), rd]).astype(np.uint32)
    lab = np.concatenate([np.zeros(3000), np.ones(2500), rl]).astype(np.uint16)
    g = rpq.load_graph(c, n, 3, src, dst, lab)
    og = oracle.Graph(n, 3, src, dst, lab)
    sample = np.arange(0, n, 7, dtype=np.uint32)
    for regex in ("a.b", "(a|b)*", "(a.b)+"):
        check(c, g, og, regex, sources=sample, mode=MODES["pull"])
