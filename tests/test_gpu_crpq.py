"""GPU parity of reverse RPQ evaluation and of CRPQ evaluation (Definition 2)
against the CPU oracle, through the C ABI."""

import numpy as np
import pytest

import oracle
from paper_2602_20748_gb300 import synth
from conftest import load_crpq_fixture, load_graph_fixture

pytestmark = pytest.mark.gpu

rpq = pytest.importorskip("paper_2602_20748_gb300.rpq")


@pytest.fixture(scope="module")
def ctx():
    return rpq.Context(device=0)


def crpq_gpu(ctx, g, n_vars, atoms, var_label=None, restrict0=None, flags=rpq.RPQ_MATERIALIZE):
    qs = [(a[0], rpq.compile_rpq(ctx, a[1]), a[2]) for a in atoms]
    r = rpq.run_crpq(ctx, g, n_vars, qs, var_label=var_label, restrict0=restrict0, flags=flags)
    info = rpq.result_info(r)
    rows = rpq.fetch_pairs(r) if flags & rpq.RPQ_MATERIALIZE else None
    return rows, info


@pytest.mark.parametrize("case", range(30))
def test_reverse_is_transposed_forward(ctx, case):
    n = 40 + 31 * (case % 5)
    L = 2 + case % 3
    src, dst, lab = synth.random_graph(n, 3 * n, L, seed=12000 + case)
    regex = synth.random_regex(13000 + case, L, max_symbols=4)
    g = rpq.load_graph(ctx, n, L, src, dst, lab)
    q = rpq.compile_rpq(ctx, regex)
    fwd = rpq.fetch_pairs(rpq.run_rpq(ctx, g, q))
    targets = np.arange(n, dtype=np.uint32) if case % 2 == 0 else np.array([0, n // 3, n - 1], np.uint32)
    rev = rpq.fetch_pairs(rpq.run_rpq(ctx, g, q, targets, flags=rpq.RPQ_MATERIALIZE | rpq.RPQ_REVERSE))
    want = sorted((int(d), int(s)) for s, d in fwd.tolist() if d in set(targets.tolist()))
    assert [tuple(r) for r in rev.tolist()] == want, regex
    # and against the oracle directly: R_G(rho) restricted to the targets, transposed
    og = oracle.Graph(n, L, src, dst, lab)
    orows = oracle.rpq(og, regex).rows
    tset = set(targets.tolist())
    want_o = sorted((int(d), int(s)) for s, d in orows.tolist() if d in tset)
    assert [tuple(r) for r in rev.tolist()] == want_o, regex


def test_handles_freed_after_context(ctx):
    c2 = rpq.Context(device=0)
    g = rpq.load_graph(c2, 10, 1, np.arange(9, dtype=np.uint32), np.arange(1, 10, dtype=np.uint32),
                       np.zeros(9, np.uint16))
    q = rpq.compile_rpq(c2, "a*")
    r = rpq.run_rpq(c2, g, q)
    c2.close()          # destroy first: deferred until the handles go
    assert rpq.result_info(r)[0] == 55
    assert len(rpq.fetch_pairs(r)) == 55
    r.free()
    g.free()
    q.free()


def test_fig1_q2(ctx):
    n, L, src, dst, lab, vl = load_graph_fixture("fig1_graph.txt")
    g = rpq.load_graph(ctx, n, L, src, dst, lab, vl)
    var_label, atoms, want = load_crpq_fixture("fig1_q2_crpq.txt")
    rows, info = crpq_gpu(ctx, g, 3, atoms, var_label=var_label)
    assert rows.tolist() == want.tolist()
    cnt, s, x = oracle.row_digest(want)
    assert info == (cnt, 3, s, x)
    rows, info2 = crpq_gpu(ctx, g, 3, atoms, var_label=var_label, flags=rpq.RPQ_COUNT_ONLY)
    assert info2 == info


def random_crpq(case, L):
    shapes = [
        (2, [(0, 1)]),
        (3, [(0, 1), (0, 2), (1, 2)]),          # triangle
        (3, [(1, 0), (1, 2), (0, 2)]),          # Q2 shape: needs a reverse atom
        (3, [(0, 1), (1, 2), (2, 0)]),          # directed cycle
        (3, [(0, 2), (1, 2)]),                  # two sources into one sink
        (4, [(0, 1), (1, 2), (2, 3), (0, 3)]),  # 4-cycle
        (2, [(0, 1), (1, 1)]),                  # self-loop atom
        (1, [(0, 0)]),                          # one variable
    ]
    nv, edges = shapes[case % len(shapes)]
    atoms = [(x, synth.random_regex(20000 + 17 * case + i, L, max_symbols=3), y) for i, (x, y) in enumerate(edges)]
    return nv, atoms


@pytest.mark.parametrize("case", range(48))
def test_random_crpq(ctx, case):
    n, L = 30 + 7 * (case % 6), 3
    src, dst, lab = synth.random_graph(n, 3 * n, L, seed=30000 + case)
    vl = synth.vertex_labels(n, 3, seed=31000 + case)
    g = rpq.load_graph(ctx, n, L, src, dst, lab, vl)
    og = oracle.Graph(n, L, src, dst, lab, vl)
    nv, atoms = random_crpq(case, L)
    var_label = None
    if case % 3 == 1:
        var_label = [int(case % 3) if i == nv - 1 else -1 for i in range(nv)]
    restrict0 = None if case % 4 != 3 else np.array([n - 1, 0, 5, 5], np.uint32)
    want = oracle.crpq(og, nv, atoms, var_label=var_label, restrict0=restrict0)
    rows, info = crpq_gpu(ctx, g, nv, atoms, var_label=var_label, restrict0=restrict0)
    assert rows.tolist() == want.rows.tolist(), atoms
    assert info[0] == len(want.rows)
    assert (info[0], info[2], info[3]) == oracle.row_digest(want.rows)
    # count only: the last variable is bound, counted and digested in one pass
    _, info_c = crpq_gpu(ctx, g, nv, atoms, var_label=var_label, restrict0=restrict0, flags=rpq.RPQ_COUNT_ONLY)
    assert (info_c[0], info_c[2], info_c[3]) == oracle.row_digest(want.rows), atoms
    # membership tests by binary search only (no bitsets), and by bitsets of
    # every non-empty row
    try:
        for frac in (2.0, 0.0):
            rpq.rpq_set_option(ctx, "crpq_bitset_frac", frac)
            rows, _ = crpq_gpu(ctx, g, nv, atoms, var_label=var_label, restrict0=restrict0)
            assert rows.tolist() == want.rows.tolist(), (frac, atoms)
            _, info_c = crpq_gpu(ctx, g, nv, atoms, var_label=var_label, restrict0=restrict0,
                                 flags=rpq.RPQ_COUNT_ONLY)
            assert (info_c[0], info_c[2], info_c[3]) == oracle.row_digest(want.rows), (frac, atoms)
    finally:
        rpq.rpq_set_option(ctx, "crpq_bitset_frac", 1 / 64)


def test_crpq_errors(ctx):
    g = rpq.load_graph(ctx, 4, 1, [0], [1], [0])
    q = rpq.compile_rpq(ctx, "a")
    with pytest.raises(rpq.RPQError) as e:     # variable 2 in no atom
        rpq.run_crpq(ctx, g, 3, [(0, q, 1)])
    assert e.value.code == rpq.RPQ_ERR_INVALID_ARG
    with pytest.raises(rpq.RPQError) as e:     # vertex labels on a graph without them
        rpq.run_crpq(ctx, g, 2, [(0, q, 1)], var_label=[0, -1])
    assert e.value.code == rpq.RPQ_ERR_INVALID_ARG


# ---------------------------------------------------------------------------
# Triangle CRPQ on R-MAT scale 22 (4,194,304 vertices, 2^26 generated edges,
# 10 labels Zipf(1.1), 5 uniform vertex labels): x -a-> y, x -b.c*-> z,
# y -d*-> z; sampled values of x.
# ---------------------------------------------------------------------------

TRIANGLE = [(0, "a", 1), (0, "b·c*", 2), (1, "d*", 2)]


@pytest.fixture(scope="module")
def rmat22(ctx):
    n = 1 << 22
    src, dst, lab = synth.rmat_graph(22, 1 << 26, 10, 1.1, seed=synth.BASE_SEED + 2)
    vl = synth.vertex_labels(n, 5, seed=synth.BASE_SEED + 2)
    return rpq.load_graph(ctx, n, 10, src, dst, lab, vl), oracle.Graph(n, 10, src, dst, lab, vl), src, lab


def test_rmat22_triangle_sampled(ctx, rmat22):
    g, og, src, lab = rmat22
    # x values with one or two a-edges (each still yields up to ~10^6 tuples:
    # a hub x yields ~10^8, beyond what the oracle finishes in seconds), plus
    # x values with no a-edge at all
    deg_a = np.bincount(src[lab == 0], minlength=1 << 22)
    rng = np.random.Generator(np.random.PCG64(23))
    sample = np.unique(np.concatenate([rng.choice(np.nonzero((deg_a >= 1) & (deg_a <= 2))[0], 12, replace=False),
                                       rng.choice(np.nonzero(deg_a == 0)[0], 4, replace=False)]))
    want = oracle.crpq(og, 3, TRIANGLE, restrict0=sample)
    rows, info = crpq_gpu(ctx, g, 3, TRIANGLE, restrict0=sample)
    assert rows.tolist() == want.rows.tolist()
    assert (info[0], info[2], info[3]) == oracle.row_digest(want.rows)
    _, info_c = crpq_gpu(ctx, g, 3, TRIANGLE, restrict0=sample, flags=rpq.RPQ_COUNT_ONLY)
    assert (info_c[0], info_c[2], info_c[3]) == oracle.row_digest(want.rows)
    try:  # binary search only
        rpq.rpq_set_option(ctx, "crpq_bitset_frac", 2.0)
        _, info_c = crpq_gpu(ctx, g, 3, TRIANGLE, restrict0=sample, flags=rpq.RPQ_COUNT_ONLY)
        assert (info_c[0], info_c[2], info_c[3]) == oracle.row_digest(want.rows)
    finally:
        rpq.rpq_set_option(ctx, "crpq_bitset_frac", 1 / 64)
    # with vertex labels on y and z
    vlab = [-1, 1, 2]
    want = oracle.crpq(og, 3, TRIANGLE, var_label=vlab, restrict0=sample)
    rows, info = crpq_gpu(ctx, g, 3, TRIANGLE, var_label=vlab, restrict0=sample)
    assert rows.tolist() == want.rows.tolist()
