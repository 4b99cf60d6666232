"""Oracle parity at the shape of the serving workload: R-MAT scale 24 (2^24
vertices, 2^28 generated edges), 16 edge labels Zipf(1.2), and the request
mix of the serving stream -- single-source RPQs (head labels), all-pairs RPQs
and triangle CRPQs (tail labels, ranks 9-16).  The oracle cannot run the full
mix at this size, so the check takes samples: single-source requests served
through rpq_server (rows of each equal the oracle's for its start vertex), a
slice of 4,096 start vertices of each all-pairs request (run_rpq_range), and
64 sampled values of x for each CRPQ (run_crpq restricted to them)."""

import concurrent.futures
import os

import numpy as np
import pytest

import oracle
from paper_2602_20748_gb300 import synth

pytestmark = pytest.mark.gpu

rpq = pytest.importorskip("paper_2602_20748_gb300.rpq")

SCALE, L = 24, 16


@pytest.fixture(scope="module")
def cfg5():
    n = 1 << SCALE
    src, dst, lab = synth.rmat_graph(SCALE, 16 << SCALE, L, 1.2, seed=synth.BASE_SEED + 5)
    t, kinds, spec = synth.serve_stream(2000.0, 1.0, L, 1.2, src, n, seed=synth.BASE_SEED + 5)
    ctx = rpq.Context(device=0)
    g = rpq.load_graph(ctx, n, L, src, dst, lab)
    og = oracle.Graph(n, L, src, dst, lab)
    del src, dst, lab
    return ctx, g, og, n, kinds, spec


def test_config5_singles_served_match_oracle(cfg5):
    ctx, g, og, n, kinds, spec = cfg5
    singles = [spec[i] for i in range(len(spec)) if kinds[i] == 1][:32]
    cache = {}
    server = rpq.Server(ctx, g, max_batch=4096)
    tickets = []
    for rx, s in singles:
        if rx not in cache:
            cache[rx] = rpq.compile_rpq(ctx, rx)
        tickets.append(server.submit_single(cache[rx], s))
    # the oracle's single-source searches side by side on the host cores
    with concurrent.futures.ThreadPoolExecutor(os.cpu_count() or 4) as ex:
        wants = list(ex.map(lambda p: oracle.pair_digest(oracle.rpq(og, p[0], sources=[p[1]], threads=1).rows), singles))
    for (rx, s), t, want in zip(singles, tickets, wants):
        rep = server.wait(t, timeout_s=300)
        assert rep["status"] == 0
        assert (rep["count"], rep["digest_sum"], rep["digest_xor"]) == want, (rx, s)
    server.close()


def test_config5_allpairs_slices_match_oracle(cfg5):
    ctx, g, og, n, kinds, spec = cfg5
    regexes = [spec[i] for i in range(len(spec)) if kinds[i] == 2][:3]
    rng = np.random.Generator(np.random.PCG64(55))
    for rx in regexes:
        b = int(rng.integers(0, n - 4096))
        q = rpq.compile_rpq(ctx, rx)
        got = rpq.fetch_pairs(rpq.run_rpq_range(ctx, g, q, b, b + 4096, rpq.RPQ_MATERIALIZE))
        want = oracle.rpq(og, rx, sources=np.arange(b, b + 4096, dtype=np.uint32)).rows
        assert np.array_equal(got, want), rx


def test_config5_crpq_sampled_x_match_oracle(cfg5):
    ctx, g, og, n, kinds, spec = cfg5
    shapes = [spec[i] for i in range(len(spec)) if kinds[i] == 3][:2]
    rng = np.random.Generator(np.random.PCG64(56))
    for l1, l2, l3, l4 in shapes:
        atoms = [(0, l1, 1), (0, f"{l2}.{l3}*", 2), (1, f"{l4}*", 2)]
        x = np.unique(rng.integers(0, n, 64)).astype(np.uint32)
        qs = [(a, rpq.compile_rpq(ctx, rx), b) for a, rx, b in atoms]
        r = rpq.run_crpq(ctx, g, 3, qs, restrict0=x, flags=rpq.RPQ_MATERIALIZE)
        got = rpq.fetch_pairs(r)
        want = oracle.crpq(og, 3, atoms, restrict0=x).rows
        assert np.array_equal(got, want), atoms
