"""Lane-mode launches: single-source RPQs with a different automaton per bit
lane, evaluated together by the multi-source engine (run_rpq_batch with
RPQ_PER_QUERY; option batch_direct sends every query there, batch_lanes caps
the lanes per launch).

Every query's reply -- the row count and digest of its own (source, y) rows
(Definition 1 for one start vertex) -- is compared with the CPU oracle's rows
for that query, and the summed work counter with the oracle's W."""

import numpy as np
import pytest

import oracle
from paper_2602_20748_gb300 import synth

pytestmark = pytest.mark.gpu

rpq = pytest.importorskip("paper_2602_20748_gb300.rpq")


def _graph(n, m, L, seed, hubs=False):
    src, dst, lab = synth.rmat_graph(15, m, L, 1.2, seed=seed)
    src %= n
    dst %= n
    if hubs:
        # rows above the chunking (128) and spill (1,024) thresholds on label a
        rng = np.random.Generator(np.random.PCG64(seed))
        src = np.concatenate([src, np.full(3000, 3, np.uint32), rng.integers(0, n, 3000).astype(np.uint32)])
        dst = np.concatenate([dst, rng.integers(0, n, 3000).astype(np.uint32), np.full(3000, 9, np.uint32)])
        lab = np.concatenate([lab, np.zeros(6000, np.uint16)])
    return src.astype(np.uint32), dst.astype(np.uint32), lab.astype(np.uint16)


def _check(c, g, og, regexes, sources):
    qs = [rpq.compile_rpq(c, r) for r in regexes]
    r = rpq.run_rpq_batch(c, g, qs, sources, flags=rpq.RPQ_PER_QUERY)
    W = 0
    for i, (rx, s) in enumerate(zip(regexes, sources)):
        want = oracle.rpq(og, rx, sources=[int(s)])
        W += want.W
        assert rpq.result_query_stats(r, i) == oracle.pair_digest(want.rows), (i, rx, int(s))
    assert rpq.result_stats(r)["product_edges"] == W
    return r


def _mix(n_q, L, src, n, seed):
    regexes, sources = synth.batch_queries(n_q, L, 1.2, src, n, seed=seed)
    # special cases: an absent label, the empty word, long automata, repeats
    regexes[1] = "z"
    regexes[2] = "z*"
    regexes[3] = "a*"
    regexes[4] = "(a.b)*"
    regexes[5] = "a.b.c.d.a.b.c.d.a"  # 10 states
    regexes[6] = "a?.b*.c?"
    sources[8] = sources[9]
    regexes[8] = regexes[9]
    sources[10] = sources[11]
    return regexes, sources


@pytest.mark.parametrize("lanes,alpha", [(4096, 16), (64, 16), (4096, 1e9), (4096, 1e-9), (200, 16)])
def test_lanes_direct_match_oracle(lanes, alpha):
    """Every query in lane mode (direct), one or several launches (64 lanes
    per launch: one 64-lane word; 200: one partly filled 256-lane group per
    launch), automatic / all bottom-up / all top-down levels."""
    c = rpq.Context(device=0)
    rpq.rpq_set_option(c, "batch_direct", 1)
    rpq.rpq_set_option(c, "batch_lanes", lanes)
    rpq.rpq_set_option(c, "alpha", alpha)
    rpq.rpq_set_option(c, "lane_alpha", alpha)  # lane-mode launches take their own
    n, L = 20000, 4
    src, dst, lab = _graph(n, 160000, L, seed=57)
    g = rpq.load_graph(c, n, L, src, dst, lab)
    og = oracle.Graph(n, L, src, dst, lab)
    regexes, sources = _mix(500, L, src, n, seed=59)
    r = _check(c, g, og, regexes, sources)
    assert rpq.result_stats(r)["evicted"] == len(regexes)


@pytest.mark.parametrize("spill_cap", [None, "3"])
def test_lanes_hub_rows_and_spill(monkeypatch, spill_cap):
    """Hubs with rows above the chunk and spill thresholds; with the spill
    capacity forced to 3 chunks per level, the chunks that do not fit are
    processed in place."""
    if spill_cap:
        monkeypatch.setenv("RPQ_SPILL_CAP", spill_cap)
    c = rpq.Context(device=0)
    rpq.rpq_set_option(c, "batch_direct", 1)
    n, L = 12000, 3
    src, dst, lab = _graph(n, 60000, L, seed=61, hubs=True)
    g = rpq.load_graph(c, n, L, src, dst, lab)
    og = oracle.Graph(n, L, src, dst, lab)
    regexes, sources = _mix(300, L, src, n, seed=63)
    sources[12:40] = 3   # from the out-hub
    sources[40:60] = 9   # from the in-hub
    _check(c, g, og, regexes, sources)


@pytest.mark.parametrize("evict,hash_", [(4, 0), (64, 0), (1024, 0), (4, 1), (64, 1), (1024, 1), (0, 1)])
def test_lanes_after_eviction_match_oracle(evict, hash_):
    """The shared per-query launch keeps light queries and evicts those that
    grow past the threshold to lane-mode launches; its visited sets are dense
    bitmaps or hash tables of 2 x threshold slots (rows counted as they are
    found; a full table evicts its query; threshold 0 with hash tables: the
    tables' default size)."""
    c = rpq.Context(device=0)
    rpq.rpq_set_option(c, "batch_evict", evict)
    rpq.rpq_set_option(c, "batch_hash", hash_)
    rpq.rpq_set_option(c, "batch_lanes", 4096)
    n, L = 20000, 4
    src, dst, lab = _graph(n, 160000, L, seed=67)
    g = rpq.load_graph(c, n, L, src, dst, lab)
    og = oracle.Graph(n, L, src, dst, lab)
    regexes, sources = _mix(400, L, src, n, seed=69)
    r = _check(c, g, og, regexes, sources)
    assert 0 < rpq.result_stats(r)["evicted"] < len(regexes)
    times = [rpq.result_query_time(r, i) for i in range(len(regexes))]
    assert min(times) >= 0 and max(times) > 0


def test_autotune_then_batch_match_oracle():
    """rpq_autotune_batch picks a representation; the tuned batch agrees with
    the oracle on every query."""
    c = rpq.Context(device=0)
    n, L = 20000, 4
    src, dst, lab = _graph(n, 160000, L, seed=71)
    g = rpq.load_graph(c, n, L, src, dst, lab)
    og = oracle.Graph(n, L, src, dst, lab)
    regexes, sources = _mix(300, L, src, n, seed=73)
    qs = [rpq.compile_rpq(c, r) for r in regexes]
    rpq.rpq_autotune_batch(c, g, qs, sources)
    assert rpq.rpq_get_option(c, "batch_lanes") == 4096
    _check(c, g, og, regexes, sources)


@pytest.mark.parametrize("by_source", [0, 1])
def test_lanes_gather_order_match_oracle(by_source):
    """Bottom-up levels of lane-mode launches gather a neighbour's frontier
    words once per (label, source state) and mask them into every target
    (by_source = 1, unions of up to 8 states), or once per union transition
    (by_source = 0); both agree with the oracle, with hub rows in the mix."""
    c = rpq.Context(device=0)
    rpq.rpq_set_option(c, "batch_direct", 1)
    rpq.rpq_set_option(c, "lane_by_source", by_source)
    rpq.rpq_set_option(c, "lane_alpha", 1e9)  # every lane-mode level bottom-up
    n, L = 12000, 3
    src, dst, lab = _graph(n, 60000, L, seed=91, hubs=True)
    g = rpq.load_graph(c, n, L, src, dst, lab)
    og = oracle.Graph(n, L, src, dst, lab)
    regexes, sources = _mix(300, L, src, n, seed=93)
    r = _check(c, g, og, regexes, sources)
    assert rpq.result_stats(r)["evicted"] == len(regexes)
