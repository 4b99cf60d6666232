"""GPU parity of run_rpq_batch (many single-source RPQs with different
expressions in one persistent launch) against the CPU oracle and against
run_rpq one query at a time, through the C ABI."""

import os

import numpy as np
import pytest

import oracle
from paper_2602_20748_gb300 import synth

pytestmark = pytest.mark.gpu

rpq = pytest.importorskip("paper_2602_20748_gb300.rpq")


@pytest.fixture(scope="module")
def ctx():
    return rpq.Context(device=0)


def oracle_batch_rows(og, regexes, sources):
    rows = []
    for i, (r, s) in enumerate(zip(regexes, sources)):
        got = oracle.rpq(og, r, sources=[int(s)]).rows
        rows.extend([i, int(d)] for d in got[:, 1])
    return np.array(rows, dtype=np.uint32).reshape(-1, 2)


@pytest.fixture(scope="module")
def er(ctx):
    src, dst, lab = synth.er_graph(1000, 5000, 4, seed=synth.BASE_SEED + 3)
    return rpq.load_graph(ctx, 1000, 4, src, dst, lab), oracle.Graph(1000, 4, src, dst, lab), src


def test_batch_matches_oracle(ctx, er):
    g, og, src = er
    regexes, sources = synth.batch_queries(300, 4, 1.2, src, 1000, seed=41)
    qs = [rpq.compile_rpq(ctx, r) for r in regexes]
    r = rpq.run_rpq_batch(ctx, g, qs, sources)
    got = rpq.fetch_pairs(r)
    want = oracle_batch_rows(og, regexes, sources)
    assert np.array_equal(got, want)
    cnt, s, x = oracle.row_digest(want)
    assert rpq.result_info(r) == (cnt, 2, s, x)
    rc = rpq.run_rpq_batch(ctx, g, qs, sources, flags=rpq.RPQ_COUNT_ONLY)
    assert rpq.result_info(rc) == rpq.result_info(r)
    # the work counter equals the sum of per-query single-source counters
    W = sum(oracle.rpq(og, rx, sources=[int(sv)]).W for rx, sv in zip(regexes, sources))
    assert rpq.result_stats(r)["product_edges"] == W


def test_batch_matches_run_rpq_per_query(ctx, er):
    g, og, src = er
    regexes, sources = synth.batch_queries(64, 4, 1.2, src, 1000, seed=43)
    qs = [rpq.compile_rpq(ctx, r) for r in regexes]
    got = rpq.fetch_pairs(rpq.run_rpq_batch(ctx, g, qs, sources))
    for i, (q, s) in enumerate(zip(qs, sources)):
        one = rpq.fetch_pairs(rpq.run_rpq(ctx, g, q, [s]))
        assert np.array_equal(got[got[:, 0] == i][:, 1], one[:, 1])


def test_batch_split_when_frontier_list_is_small(er):
    old = os.environ.get("RPQ_BATCH_LIST_CAP")
    os.environ["RPQ_BATCH_LIST_CAP"] = "2000"
    try:
        c2 = rpq.Context(device=0)
    finally:
        if old is None:
            del os.environ["RPQ_BATCH_LIST_CAP"]
        else:
            os.environ["RPQ_BATCH_LIST_CAP"] = old
    g0, og, src = er
    s0, d0, l0 = synth.er_graph(1000, 5000, 4, seed=synth.BASE_SEED + 3)
    g = rpq.load_graph(c2, 1000, 4, s0, d0, l0)
    regexes, sources = synth.batch_queries(200, 4, 1.2, src, 1000, seed=47)
    qs = [rpq.compile_rpq(c2, r) for r in regexes]
    got = rpq.fetch_pairs(rpq.run_rpq_batch(c2, g, qs, sources))
    assert np.array_equal(got, oracle_batch_rows(og, regexes, sources))


def test_batch_autotune_and_edge_cases(ctx, er):
    g, og, src = er
    regexes, sources = synth.batch_queries(100, 4, 1.2, src, 1000, seed=53)
    regexes[3] = "z"          # label absent from the graph: empty result
    regexes[4] = "a*"         # empty word: (s, s) at least
    qs = [rpq.compile_rpq(ctx, r) for r in regexes]
    t, k = rpq.rpq_autotune_batch(ctx, g, qs, sources)
    assert t in (128, 256, 512) and k in (1024, 2048, 4096)
    got = rpq.fetch_pairs(rpq.run_rpq_batch(ctx, g, qs, sources))
    assert np.array_equal(got, oracle_batch_rows(og, regexes, sources))
    assert len(got[got[:, 0] == 3]) == 0
    r = rpq.run_rpq_batch(ctx, g, [], np.zeros(0, np.uint32))
    assert rpq.result_info(r)[0] == 0
    with pytest.raises(rpq.RPQError) as e:
        rpq.run_rpq_batch(ctx, g, qs[:1], [1000])
    assert e.value.code == rpq.RPQ_ERR_INVALID_ARG


@pytest.mark.parametrize("evict,alpha,multi", [(0, 16, 0), (40, 16, 0), (65536, 16, 0), (40, 16, 1), (40, 1e9, 1),
                                               (40, 1e-9, 1)])
def test_batch_per_query_matches_standalone(evict, alpha, multi):
    """RPQ_PER_QUERY: every query's row count and digest equal run_rpq's for
    that query alone, whether it stays in the shared launch or is evicted and
    evaluated by the multi-source engine (threshold 40 evicts most queries,
    0 none; with multi = 1 small automaton groups share multi-automaton
    launches); alpha 1e9 / 1e-9 makes every level bottom-up / top-down.  The
    work counter stays exact."""
    c = rpq.Context(device=0)
    rpq.rpq_set_option(c, "batch_evict", evict)
    rpq.rpq_set_option(c, "alpha", alpha)
    rpq.rpq_set_option(c, "batch_multi", multi)
    n = 20000
    src, dst, lab = synth.rmat_graph(15, 8 * n, 4, 1.2, seed=57)
    src %= n
    dst %= n
    g = rpq.load_graph(c, n, 4, src, dst, lab)
    regexes, sources = synth.batch_queries(400, 4, 1.2, src, n, seed=59)
    regexes[5] = "z"  # label absent: empty
    sources[7] = sources[8]  # duplicate start vertex
    regexes[7] = regexes[8]
    qs = [rpq.compile_rpq(c, r) for r in regexes]
    r = rpq.run_rpq_batch(c, g, qs, sources, flags=rpq.RPQ_PER_QUERY)
    tot = [0, 0, 0]
    W = 0
    for i, (q, s) in enumerate(zip(qs, sources)):
        one = rpq.run_rpq(c, g, q, [s], flags=rpq.RPQ_COUNT_ONLY)
        cnt, _, hs, hx = rpq.result_info(one)
        W += rpq.result_stats(one)["product_edges"]
        one.free()
        assert rpq.result_query_stats(r, i) == (cnt, hs, hx), (i, regexes[i])
        tot[0] += cnt
        tot[1] = (tot[1] + hs) & 0xFFFFFFFFFFFFFFFF
        tot[2] ^= hx
    assert rpq.result_info(r) == (tot[0], 2, tot[1], tot[2])
    assert rpq.result_stats(r)["product_edges"] == W
    with pytest.raises(rpq.RPQError):
        rpq.result_query_stats(r, 400)
    # a few queries against the oracle directly
    og = oracle.Graph(n, 4, src, dst, lab)
    for i in (0, 5, 7, 123):
        want = oracle.rpq(og, regexes[i], sources=[int(sources[i])]).rows
        assert rpq.result_query_stats(r, i) == oracle.pair_digest(want)


def test_batch_rmat22_sampled(ctx):
    """4,096 queries on R-MAT scale 22 (2^26 edges, 8 labels Zipf 1.2),
    sources proportional to out-degree; sampled queries row by row."""
    n = 1 << 22
    src, dst, lab = synth.rmat_graph(22, 1 << 26, 8, 1.2, seed=synth.BASE_SEED + 4)
    g = rpq.load_graph(ctx, n, 8, src, dst, lab)
    og = oracle.Graph(n, 8, src, dst, lab)
    regexes, sources = synth.batch_queries(4096, 8, 1.2, src, n, seed=synth.BASE_SEED + 4)
    qs = [rpq.compile_rpq(ctx, r) for r in regexes]
    r = rpq.run_rpq_batch(ctx, g, qs, sources)
    got = rpq.fetch_pairs(r)
    rng = np.random.Generator(np.random.PCG64(3))
    for i in rng.choice(4096, 6, replace=False):
        want = oracle.rpq(og, regexes[i], sources=[int(sources[i])]).rows[:, 1]
        assert np.array_equal(got[got[:, 0] == i][:, 1], want), regexes[i]


def test_batch_spill_capacity_overflow():
    """As for the all-pairs engine: with the long-row chunk capacity forced
    down to 3, rows that do not fit are processed in place."""
    old = os.environ.get("RPQ_SPILL_CAP")
    os.environ["RPQ_SPILL_CAP"] = "3"
    try:
        c3 = rpq.Context(device=0)
    finally:
        if old is None:
            del os.environ["RPQ_SPILL_CAP"]
        else:
            os.environ["RPQ_SPILL_CAP"] = old
    n = 6000
    rs, rd, rl = synth.random_graph(n, 12000, 2, seed=91)
    src = np.concatenate([np.repeat(np.arange(10, dtype=np.uint32), 2500), rs]).astype(np.uint32)
    dst = np.concatenate([synth.random_graph(n, 25000, 1, seed=92)[1], rd]).astype(np.uint32)
    lab = np.concatenate([np.zeros(25000, np.uint16), rl]).astype(np.uint16)
    g = rpq.load_graph(c3, n, 2, src, dst, lab)
    og = oracle.Graph(n, 2, src, dst, lab)
    regexes = ["a.b*", "(a|b)+", "a", "a.a", "b*.a"] * 12
    sources = np.array([i % 10 if i % 3 else 100 + i for i in range(len(regexes))], np.uint32)
    qs = [rpq.compile_rpq(c3, r) for r in regexes]
    got = rpq.fetch_pairs(rpq.run_rpq_batch(c3, g, qs, sources))
    assert np.array_equal(got, oracle_batch_rows(og, regexes, sources))
