"""The serving loop: every request's reply (row count and digest) equals the
CPU oracle's result for that request -- Definition 1 rows (source, y) for a
single-source request, all (x, y) rows for an all-pairs request, Definition 2
tuples for a CRPQ -- whether it is served alone or in a mix of many
concurrent requests of all kinds, through the C ABI.  Single-source requests
are admitted into a running serving launch; those that grow past the
eviction threshold are finished in lane-mode launches."""

import time

import numpy as np
import pytest

import oracle
from paper_2602_20748_gb300 import synth

pytestmark = pytest.mark.gpu

rpq = pytest.importorskip("paper_2602_20748_gb300.rpq")

CRPQS = [[(0, "a", 1), (0, "b.c*", 2), (1, "d*", 2)],
         [(0, "e", 1), (1, "f*", 2), (0, "(e|f)", 2)]]
ALLPAIRS = ("f*", "e.f*", "(e|f)+")


@pytest.fixture(scope="module")
def setup():
    ctx = rpq.Context(device=0)
    n = 3000
    src, dst, lab = synth.rmat_graph(12, 6 * n, 6, 1.2, seed=61)
    src %= n
    dst %= n
    vl = synth.vertex_labels(n, 3, seed=62)
    g = rpq.load_graph(ctx, n, 6, src, dst, lab, vl)
    og = oracle.Graph(n, 6, src, dst, lab, vl)
    regexes, sources = synth.batch_queries(240, 6, 1.2, src, n, seed=63)
    return ctx, g, og, n, regexes, sources


def oracle_reply(og, kind, spec):
    if kind == "single":
        regex, s = spec
        return oracle.pair_digest(oracle.rpq(og, regex, sources=[s]).rows)
    if kind == "allpairs":
        return oracle.pair_digest(oracle.rpq(og, spec).rows)
    return oracle.row_digest(oracle.crpq(og, 3, spec).rows)


def submit(server, ctx, cache, kind, spec):
    def comp(rx):
        if rx not in cache:
            cache[rx] = rpq.compile_rpq(ctx, rx)
        return cache[rx]

    if kind == "single":
        return server.submit_single(comp(spec[0]), spec[1])
    if kind == "allpairs":
        return server.submit_allpairs(comp(spec))
    return server.submit_crpq(3, [(x, comp(rx), y) for x, rx, y in spec])


def test_served_results_equal_oracle_alone_and_in_the_mix(setup):
    ctx, g, og, n, regexes, sources = setup
    work = [("single", (rx, int(s))) for rx, s in zip(regexes, sources)]
    work += [("allpairs", rx) for rx in ALLPAIRS] + [("crpq", c) for c in CRPQS]
    want = [oracle_reply(og, k, p) for k, p in work]
    cache = {}
    # in the mix: everything submitted at once, interleaved
    server = rpq.Server(ctx, g, max_batch=64)
    order = np.random.Generator(np.random.PCG64(5)).permutation(len(work))
    tickets = {int(i): submit(server, ctx, cache, *work[i]) for i in order}
    for i, t in tickets.items():
        rep = server.wait(t, timeout_s=120)
        assert rep["status"] == 0, work[i]
        assert (rep["count"], rep["digest_sum"], rep["digest_xor"]) == want[i], work[i]
    launches, admitted = server.stats()
    # every single-source request passed through the serving launch, and they
    # shared launches (a request that arrives while one runs joins it)
    assert admitted == len(regexes) and launches < len(regexes)
    info = server.info()
    assert info["launches"] == launches and info["admitted"] == admitted and info["graph"] == 1
    server.close()
    # alone: one request at a time
    server = rpq.Server(ctx, g, max_batch=64)
    for i in range(0, len(work), 25):
        rep = server.wait(submit(server, ctx, cache, *work[i]), timeout_s=120)
        assert (rep["count"], rep["digest_sum"], rep["digest_xor"]) == want[i], work[i]
    server.close()


def test_stream_with_evictions_matches_oracle():
    """Single-source requests arriving over time on a 20,000-vertex graph:
    many outgrow the serving launch's 4,096-product-vertex threshold and are
    finished in lane-mode launches; every reply equals the oracle's."""
    ctx = rpq.Context(device=0)
    n, L = 20000, 4
    src, dst, lab = synth.rmat_graph(15, 8 * n, L, 1.2, seed=81)
    src %= n
    dst %= n
    g = rpq.load_graph(ctx, n, L, src, dst, lab)
    og = oracle.Graph(n, L, src, dst, lab)
    regexes, sources = synth.batch_queries(400, L, 1.2, src, n, seed=83)
    regexes[0], regexes[1] = "a*", "z"
    cache = {}
    server = rpq.Server(ctx, g, max_batch=256)
    tickets = []
    for i, (rx, s) in enumerate(zip(regexes, sources)):
        tickets.append(submit(server, ctx, cache, "single", (rx, int(s))))
        if i % 50 == 49:
            time.sleep(0.002)  # later requests arrive while earlier ones run
    evicted_possible = 0
    for i, t in enumerate(tickets):
        rep = server.wait(t, timeout_s=120)
        want = oracle.rpq(og, regexes[i], sources=[int(sources[i])])
        evicted_possible += want.N > 4096
        assert rep["status"] == 0
        assert (rep["count"], rep["digest_sum"], rep["digest_xor"]) == oracle.pair_digest(want.rows), i
    assert evicted_possible > 0
    info = server.info()
    assert info["lane_requests"] >= evicted_possible and info["lane_launches"] > 0
    server.close()


def test_set_option(setup):
    c2 = rpq.Context(device=0)
    rpq.rpq_set_option(c2, "grid_share", 0.5)
    rpq.rpq_set_option(c2, "alpha", 8)
    with pytest.raises(rpq.RPQError):
        rpq.rpq_set_option(c2, "no_such_option", 1)
    with pytest.raises(rpq.RPQError):
        rpq.rpq_set_option(c2, "grid_share", 2)


def test_cancel_stops_queued_and_running_requests(setup):
    ctx, g, og, n, regexes, sources = setup
    cache = {}
    server = rpq.Server(ctx, g, max_batch=64)
    bulk = [submit(server, ctx, cache, "allpairs", "(a|b|c|d|e|f)*") for _ in range(20)]
    singles = [submit(server, ctx, cache, "single", (rx, int(s))) for rx, s in zip(regexes[:50], sources[:50])]
    server.cancel()
    statuses = [server.wait(t, timeout_s=120)["status"] for t in bulk + singles]
    assert all(s in (0, rpq.RPQ_ERR_CANCELLED) for s in statuses)
    assert statuses[len(bulk) - 1] == rpq.RPQ_ERR_CANCELLED
    # the server keeps serving after a cancel
    want = oracle_reply(og, "single", (regexes[0], int(sources[0])))
    rep = server.wait(submit(server, ctx, cache, "single", (regexes[0], int(sources[0]))), timeout_s=120)
    assert rep["status"] == 0 and (rep["count"], rep["digest_sum"], rep["digest_xor"]) == want
    server.close()
