"""The serving loop: every request's reply (row count and digest) equals the
standalone call's, whether the request is served alone or in a mix with many
concurrent requests of all kinds, through the C ABI."""

import numpy as np
import pytest

from paper_2602_20748_gb300 import synth

pytestmark = pytest.mark.gpu

rpq = pytest.importorskip("paper_2602_20748_gb300.rpq")


@pytest.fixture(scope="module")
def setup():
    ctx = rpq.Context(device=0)
    n = 3000
    src, dst, lab = synth.rmat_graph(12, 6 * n, 6, 1.2, seed=61)
    src %= n
    dst %= n
    vl = synth.vertex_labels(n, 3, seed=62)
    g = rpq.load_graph(ctx, n, 6, src, dst, lab, vl)
    regexes, sources = synth.batch_queries(240, 6, 1.2, src, n, seed=63)
    return ctx, g, n, regexes, sources


def standalone(ctx, g, kind, payload):
    if kind == "single":
        q, s = payload
        r = rpq.run_rpq(ctx, g, q, [s], flags=rpq.RPQ_COUNT_ONLY)
    elif kind == "allpairs":
        r = rpq.run_rpq(ctx, g, payload, flags=rpq.RPQ_COUNT_ONLY)
    else:
        r = rpq.run_crpq(ctx, g, 3, payload, flags=rpq.RPQ_COUNT_ONLY)
    c, _, s, x = rpq.result_info(r)
    return c, s, x


def test_served_results_equal_standalone_alone_and_in_the_mix(setup):
    ctx, g, n, regexes, sources = setup
    qs = [rpq.compile_rpq(ctx, r) for r in regexes]
    ap = [rpq.compile_rpq(ctx, r) for r in ("f*", "e.f*", "(e|f)+")]
    crpqs = [[(0, rpq.compile_rpq(ctx, "a"), 1), (0, rpq.compile_rpq(ctx, "b.c*"), 2),
              (1, rpq.compile_rpq(ctx, "d*"), 2)],
             [(0, rpq.compile_rpq(ctx, "e"), 1), (1, rpq.compile_rpq(ctx, "f*"), 2),
              (0, rpq.compile_rpq(ctx, "(e|f)"), 2)]]
    work = [("single", (q, int(s))) for q, s in zip(qs, sources)]
    work += [("allpairs", q) for q in ap] + [("crpq", c) for c in crpqs]
    want = [standalone(ctx, g, k, p) for k, p in work]

    def submit(server, k, p):
        if k == "single":
            return server.submit_single(*p)
        if k == "allpairs":
            return server.submit_allpairs(p)
        return server.submit_crpq(3, p)

    # in the mix: everything submitted at once, interleaved
    server = rpq.Server(ctx, g, max_batch=64)
    order = np.random.Generator(np.random.PCG64(5)).permutation(len(work))
    tickets = {int(i): submit(server, *work[i]) for i in order}
    for i, t in tickets.items():
        rep = server.wait(t, timeout_s=120)
        assert rep["status"] == 0
        assert (rep["count"], rep["digest_sum"], rep["digest_xor"]) == want[i], work[i][0]
    batches, carried = server.stats()
    assert carried == len(regexes) and batches < len(regexes)  # singles were batched
    server.close()
    # alone: one request at a time
    server = rpq.Server(ctx, g, max_batch=64)
    for i in range(0, len(work), 25):
        rep = server.wait(submit(server, *work[i]), timeout_s=120)
        assert (rep["count"], rep["digest_sum"], rep["digest_xor"]) == want[i]
    server.close()


def test_set_option(setup):
    ctx = setup[0]
    c2 = rpq.Context(device=0)
    rpq.rpq_set_option(c2, "grid_share", 0.5)
    rpq.rpq_set_option(c2, "alpha", 8)
    with pytest.raises(rpq.RPQError):
        rpq.rpq_set_option(c2, "no_such_option", 1)
    with pytest.raises(rpq.RPQError):
        rpq.rpq_set_option(c2, "grid_share", 2)


def test_cancel_stops_queued_and_running_requests(setup):
    ctx, g, n, regexes, sources = setup
    ap = rpq.compile_rpq(ctx, "(a|b|c|d|e|f)*")
    q = rpq.compile_rpq(ctx, regexes[0])
    want = standalone(ctx, g, "single", (q, int(sources[0])))
    server = rpq.Server(ctx, g, max_batch=64)
    bulk = [server.submit_allpairs(ap) for _ in range(20)]
    server.cancel()
    statuses = [server.wait(t, timeout_s=120)["status"] for t in bulk]
    assert all(s in (0, rpq.RPQ_ERR_CANCELLED) for s in statuses)
    assert statuses[-1] == rpq.RPQ_ERR_CANCELLED
    # the server keeps serving after a cancel
    rep = server.wait(server.submit_single(q, int(sources[0])), timeout_s=120)
    assert rep["status"] == 0 and (rep["count"], rep["digest_sum"], rep["digest_xor"]) == want
    server.close()
