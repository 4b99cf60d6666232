"""Start-in-the-middle plan (run_rpq_middle): rho = alpha . beta evaluated by
materializing R(beta) first and joining it with alpha as one extra edge label
(Section 2.3 WavePlan A3, executed as A5 of Section 6.3).  The plan changes
only the exploration order, so its rows must equal the oracle's rows of
alpha . beta (Definition 1) exactly."""

import numpy as np
import pytest

import oracle
from conftest import load_graph_fixture, load_rows
from paper_2602_20748_gb300 import synth

pytestmark = pytest.mark.gpu

rpq = pytest.importorskip("paper_2602_20748_gb300.rpq")


@pytest.fixture(scope="module")
def ctx():
    return rpq.Context(device=0)


def _middle_rows(ctx, g, a, b, sources=None, flags=None):
    qa, qb = rpq.compile_rpq(ctx, a), rpq.compile_rpq(ctx, b)
    r = rpq.run_rpq_middle(ctx, g, qa, qb, sources, flags=rpq.RPQ_MATERIALIZE if flags is None else flags)
    return rpq.fetch_pairs(r)


def test_fig1_abcstar_from_the_middle(ctx):
    """Q1 = abc* on Figure 1 through both split points gives the 13 pairs the
    paper lists (the footnote of the Introduction)."""
    n, L, src, dst, lab, _ = load_graph_fixture("fig1_graph.txt")
    g = rpq.load_graph(ctx, n, L, src, dst, lab)
    want = load_rows("fig1_q1_abcstar.txt")
    for a, b in (("a", "b.c*"), ("a.b", "c*"), ("a.b.c*", "c*")):
        got = _middle_rows(ctx, g, a, b)
        assert np.array_equal(got, want), (a, b)


def test_er_config_full(ctx):
    src, dst, lab = synth.er_graph(1000, 5000, 4, seed=synth.BASE_SEED)
    g = rpq.load_graph(ctx, 1000, 4, src, dst, lab)
    og = oracle.Graph(1000, 4, src, dst, lab)
    want = oracle.rpq(og, "a.b.c*").rows
    for flags in (rpq.RPQ_MATERIALIZE, rpq.RPQ_MATERIALIZE | rpq.RPQ_FORCE_PUSH,
                  rpq.RPQ_MATERIALIZE | rpq.RPQ_FORCE_PULL):
        assert np.array_equal(_middle_rows(ctx, g, "a", "b.c*", flags=flags), want)
    # count only: the same count and digest
    qa, qb = rpq.compile_rpq(ctx, "a"), rpq.compile_rpq(ctx, "b.c*")
    r = rpq.run_rpq_middle(ctx, g, qa, qb, flags=rpq.RPQ_COUNT_ONLY)
    c, _, hs, hx = rpq.result_info(r)
    assert (c, hs, hx) == oracle.pair_digest(want)


@pytest.mark.parametrize("case", range(24))
def test_random_splits_match_oracle(ctx, case):
    n = 60 + 37 * case
    src, dst, lab = synth.random_graph(n, 4 * n, 3, seed=900 + case)
    g = rpq.load_graph(ctx, n, 3, src, dst, lab)
    og = oracle.Graph(n, 3, src, dst, lab)
    a = synth.random_regex(1000 + case, 3, max_symbols=3)
    b = synth.random_regex(2000 + case, 3, max_symbols=3)
    want = oracle.rpq(og, f"({a}).({b})").rows
    assert np.array_equal(_middle_rows(ctx, g, a, b), want), (a, b)
    sources = np.unique(np.random.Generator(np.random.PCG64(case)).integers(0, n, 7)).astype(np.uint32)
    want_s = oracle.rpq(og, f"({a}).({b})", sources=sources).rows
    assert np.array_equal(_middle_rows(ctx, g, a, b, sources), want_s), (a, b)


def test_empty_word_and_absent_labels(ctx):
    src, dst, lab = synth.er_graph(500, 2500, 4, seed=synth.BASE_SEED + 3)
    g = rpq.load_graph(ctx, 500, 4, src, dst, lab)
    og = oracle.Graph(500, 4, src, dst, lab)
    for a, b in (("a*", "b*"), ("a?", "c"), ("z", "a*"), ("a", "z*"), ("a*.b", "z")):
        want = oracle.rpq(og, f"({a}).({b})").rows
        assert np.array_equal(_middle_rows(ctx, g, a, b), want), (a, b)


def test_rmat_batch_equals_forward(ctx):
    """R-MAT scale 16: the middle plan from a batch of 4,096 start vertices
    equals the forward plan's rows (run_rpq of alpha . beta), and sampled
    start vertices equal the oracle's."""
    n = 1 << 16
    src, dst, lab = synth.rmat_graph(16, 16 * n, 8, 1.2, seed=synth.BASE_SEED + 1)
    g = rpq.load_graph(ctx, n, 8, src, dst, lab)
    sources = np.arange(8192, 8192 + 4096, dtype=np.uint32)
    for a, b in (("a", "b.c*"), ("a.b*", "c"), ("(a|b)+", "c")):
        q = rpq.compile_rpq(ctx, f"({a}).({b})")
        want = rpq.fetch_pairs(rpq.run_rpq(ctx, g, q, sources))
        got = _middle_rows(ctx, g, a, b, sources)
        assert np.array_equal(got, want), (a, b)
    og = oracle.Graph(n, 8, src, dst, lab)
    few = sources[::512]
    want = oracle.rpq(og, "a.b.c*", sources=few).rows
    assert np.array_equal(_middle_rows(ctx, g, "a", "b.c*", few), want)
