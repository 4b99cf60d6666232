"""Pins for the CPU oracle against facts fixed outside the oracle itself:
the paper's worked example (Figure 1 / Table 1, Section 1 footnote, the
algebra example of Section 2.2, the Q2 CRPQ), a second algorithm
(boolean-matrix algebra, oracle/algebra.py), closed forms from graph theory,
and invariants of regular languages.  CPU only."""

import itertools

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import oracle
from oracle import algebra
from paper_2602_20748_gb300 import synth
from conftest import load_crpq_fixture, load_graph_fixture, load_rows


@pytest.fixture(scope="module")
def fig1():
    n, L, src, dst, lab, vl = load_graph_fixture("fig1_graph.txt")
    return n, L, src, dst, lab, vl, oracle.Graph(n, L, src, dst, lab, vl)


def as_set(rows):
    return {tuple(int(x) for x in r) for r in rows}


# --------------------------------------------------------------------------
# Worked example of the paper
# --------------------------------------------------------------------------

def test_fig1_q1_abcstar_matches_paper(fig1):
    """Section 1 footnote: Q1 = abc* returns exactly 13 pairs."""
    n, L, src, dst, lab, vl, g = fig1
    want = load_rows("fig1_q1_abcstar.txt")
    got = oracle.rpq(g, "abc*")
    assert got.rows.tolist() == want.tolist()
    assert got.automaton_mismatch == 0
    assert algebra.rpq_pairs(n, L, src, dst, lab, "abc*").tolist() == want.tolist()


def test_fig1_label_a_relation(fig1):
    """Section 2.2: the relation of label a is {(0,1),(0,3),(0,6),(2,5),(7,5)}."""
    g = fig1[-1]
    assert oracle.rpq(g, "a").rows.tolist() == load_rows("fig1_a_relation.txt").tolist()


def test_fig1_single_sources(fig1):
    """From v0: 9 pairs; v2: 2; v7: 2 (counted from the Section 1 footnote).
    Single-source equals the all-pairs result restricted to that source."""
    g = fig1[-1]
    allp = oracle.rpq(g, "abc*").rows
    for s, k in [(0, 9), (2, 2), (7, 2), (5, 0), (13, 0)]:
        r = oracle.rpq(g, "abc*", sources=[s]).rows
        assert len(r) == k
        assert r.tolist() == allp[allp[:, 0] == s].tolist()


def test_fig1_four_hop_witness(fig1):
    """Section 3: (v0, v9) is reached by the 4-hop path 0->3->12->13->9 (abcc);
    with abc (exactly one c) v9 is not reachable from v0, with abcc it is."""
    g = fig1[-1]
    assert (0, 9) not in as_set(oracle.rpq(g, "abc", sources=[0]).rows)
    assert (0, 9) in as_set(oracle.rpq(g, "abcc", sources=[0]).rows)


def test_fig1_min_dfa_shape():
    """Section 4.1 example: the plan for abc* is q0 -a-> q1 -b-> q2 with a
    c self-loop on the final state q2."""
    k, fin, nxt = oracle.dfa("abc*", 3)
    assert k == 3
    assert fin.tolist() == [False, False, True]
    assert nxt.tolist() == [[1, -1, -1], [-1, 2, -1], [-1, -1, 2]]


def test_abcd_has_five_states():
    """Section 3, Challenge 2: for Q4 = abcd the automaton has |Q| = 5."""
    assert oracle.dfa("abcd", 4)[0] == 5


@pytest.mark.parametrize("regex,states", [("a*", 1), ("(a|b)+.c", 3), ("a.b*.c", 3), ("(a.b)*", 2),
                                          ("a.b.c*", 3), ("a?b*", 2), ("a*b*", 2)])
def test_min_dfa_state_counts(regex, states):
    """Textbook minimal partial DFAs of small expressions."""
    assert oracle.dfa(regex, 4)[0] == states


def test_q2_crpq_matches_paper(fig1):
    """Section 1: Q2 on (u2,u3,u4) = {(10,0,10),(10,0,12),(12,0,10),(12,0,12)}
    (query graph reconstructed, see the fixture header)."""
    g = fig1[-1]
    var_label, atoms, want = load_crpq_fixture("fig1_q2_crpq.txt")
    got = oracle.crpq(g, 3, atoms, var_label=var_label)
    assert got.rows.tolist() == want.tolist()


def test_q2_atom_blocks(fig1):
    """Section 2.4: the ab result block P'_0 from A to D is {(0,10),(0,12)};
    the D x D block of c* holds 16 pairs."""
    n, L, src, dst, lab, vl, g = fig1
    ab = oracle.rpq(g, "ab").rows
    a_to_d = [r for r in ab.tolist() if vl[r[0]] == 0 and vl[r[1]] == 3]
    assert a_to_d == [[0, 10], [0, 12]]
    cs = oracle.rpq(g, "c*").rows
    dd = [r for r in cs.tolist() if vl[r[0]] == 3 and vl[r[1]] == 3]
    assert len(dd) == 16


def test_splitmix64_published_outputs():
    """SplitMix64 (Steele, Lea, Flood 2014): first output from state 0 is
    0xE220A8397B1DCDAF; from seed 1234567 the outputs begin
    6457827717110365317, 3203168211198807973."""
    assert oracle.splitmix64(0) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64(1234567) == 6457827717110365317
    assert oracle.splitmix64(1234567 + oracle.GOLDEN_GAMMA) == 3203168211198807973
    arr = oracle.splitmix64(np.array([0, 1234567], dtype=np.uint64))
    assert arr.tolist() == [0xE220A8397B1DCDAF, 6457827717110365317]


# --------------------------------------------------------------------------
# Closed forms
# --------------------------------------------------------------------------

def test_star_on_cycle_gives_n_squared():
    n = 37
    src = np.arange(n, dtype=np.uint32)
    dst = (src + 1) % n
    g = oracle.Graph(n, 1, src, dst, np.zeros(n, np.uint16))
    r = oracle.rpq(g, "a*")
    assert len(r.rows) == n * n
    # one state, every product vertex reached from every source, deg 1 each
    assert r.W == n * n and r.N == n * n


def test_star_on_path_gives_triangle_number():
    n = 50
    src = np.arange(n - 1, dtype=np.uint32)
    g = oracle.Graph(n, 1, src, src + 1, np.zeros(n - 1, np.uint16))
    assert len(oracle.rpq(g, "a*").rows) == n * (n + 1) // 2
    assert len(oracle.rpq(g, "a+").rows) == n * (n - 1) // 2


def test_single_label_is_deduplicated_edge_set():
    src, dst, lab = synth.random_graph(60, 900, 3, seed=11)
    g = oracle.Graph(60, 3, src, dst, lab)
    want = sorted({(int(s), int(d)) for s, d, l in zip(src, dst, lab) if l == 1})
    r = oracle.rpq(g, "b")
    assert [tuple(x) for x in r.rows.tolist()] == want
    # minimal DFA q0 -b-> q1; only q0 has a transition: W = |E_b|
    assert r.W == len(want)
    edges = {(int(s), int(d), int(l)) for s, d, l in zip(src, dst, lab)}
    assert g.n_edges == len(edges)


def test_plus_on_dag_is_transitive_closure():
    """On a DAG, R(a+) is the transitive closure (scipy reachability)."""
    n = 80
    st = np.random.Generator(np.random.PCG64(5)).bit_generator.random_raw(400)
    u = (st % n).astype(np.int64)
    v = ((st >> np.uint64(20)) % n).astype(np.int64)
    keep = u < v
    src, dst = u[keep].astype(np.uint32), v[keep].astype(np.uint32)
    g = oracle.Graph(n, 1, src, dst, np.zeros(len(src), np.uint16))
    m = sp.csr_matrix((np.ones(len(src)), (src, dst)), shape=(n, n))
    dist = csg.shortest_path(m, directed=True, unweighted=True)
    want = {(i, j) for i in range(n) for j in range(n) if i != j and np.isfinite(dist[i, j])}
    assert as_set(oracle.rpq(g, "a+").rows) == want


def test_work_counter_star_closed_form():
    """For l*, W = sum over s, over v reachable by l-paths (incl. s), of deg_l(v)."""
    src, dst, lab = synth.random_graph(70, 260, 2, seed=3)
    g = oracle.Graph(70, 2, src, dst, lab)
    e = {(int(s), int(d)) for s, d, l in zip(src, dst, lab) if l == 0}
    deg = np.zeros(70, np.int64)
    for s, _ in e:
        deg[s] += 1
    m = sp.csr_matrix((np.ones(len(e)), ([a for a, _ in e], [b for _, b in e])), shape=(70, 70))
    dist = csg.shortest_path(m, directed=True, unweighted=True)
    want = int(sum(deg[v] for s in range(70) for v in range(70) if np.isfinite(dist[s, v])))
    assert oracle.rpq(g, "a*").W == want


# --------------------------------------------------------------------------
# Second algorithm: boolean-matrix algebra
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case", range(120))
def test_random_against_algebra(case):
    n = 6 + case % 23
    m = n * (1 + case % 4)
    L = 2 + case % 3
    src, dst, lab = synth.random_graph(n, m, L, seed=1000 + case)
    regex = synth.random_regex(2000 + case, L)
    g = oracle.Graph(n, L, src, dst, lab)
    got = oracle.rpq(g, regex)
    want = algebra.rpq_pairs(n, L, src, dst, lab, regex)
    assert got.rows.tolist() == want.tolist(), regex
    assert got.automaton_mismatch == 0


def test_epsilon_gives_identity_including_isolated():
    n = 10
    g = oracle.Graph(n, 2, np.array([0, 1], np.uint32), np.array([1, 2], np.uint32), np.array([0, 0], np.uint16))
    r = as_set(oracle.rpq(g, "b*").rows)
    assert r == {(v, v) for v in range(n)}
    r = as_set(oracle.rpq(g, "a?").rows)
    assert r == {(v, v) for v in range(n)} | {(0, 1), (1, 2)}


def test_label_absent_from_graph_matches_nothing():
    g = oracle.Graph(4, 2, np.array([0], np.uint32), np.array([1], np.uint32), np.array([0], np.uint16))
    assert len(oracle.rpq(g, "z").rows) == 0
    assert len(oracle.rpq(g, "a.z").rows) == 0
    assert as_set(oracle.rpq(g, "a|z").rows) == {(0, 1)}


@pytest.mark.parametrize("bad", ["a|", "(a", "*a", "a)", "", "a**(", "A"])
def test_parse_errors(bad):
    g = oracle.Graph(2, 1, np.array([0], np.uint32), np.array([1], np.uint32), np.array([0], np.uint16))
    with pytest.raises(oracle.OracleError) as e:
        oracle.rpq(g, bad)
    assert e.value.code == -2


def test_label_names_table():
    names = ["knows", "likes", "replyOf"]
    g = oracle.Graph(3, 3, np.array([0, 1], np.uint32), np.array([1, 2], np.uint32), np.array([0, 2], np.uint16))
    assert as_set(oracle.rpq(g, "knows.replyOf*", names=names).rows) == {(0, 1), (0, 2)}
    with pytest.raises(oracle.OracleError) as e:
        oracle.rpq(g, "hates", names=names)
    assert e.value.code == -3


# --------------------------------------------------------------------------
# Invariants
# --------------------------------------------------------------------------

def _rev(tree):
    k = tree[0]
    if k == "L":
        return chr(ord("a") + tree[1])
    if k == "cat":
        return f"({_rev(tree[2])}).({_rev(tree[1])})"
    if k == "alt":
        return f"({_rev(tree[1])})|({_rev(tree[2])})"
    op = {"star": "*", "plus": "+", "opt": "?"}[k]
    return f"({_rev(tree[1])}){op}"


@pytest.mark.parametrize("case", range(25))
def test_invariants(case):
    n, L = 25, 3
    src, dst, lab = synth.random_graph(n, 70, L, seed=500 + case)
    g = oracle.Graph(n, L, src, dst, lab)
    r1 = synth.random_regex(600 + case, L, max_symbols=3)
    r2 = synth.random_regex(700 + case, L, max_symbols=3)
    R = lambda x: as_set(oracle.rpq(g, x).rows)
    A, B = R(r1), R(r2)
    # union
    assert R(f"({r1})|({r2})") == A | B
    # concatenation = relational composition
    comp = {(x, z) for (x, y) in A for (y2, z) in B if y == y2}
    assert R(f"({r1}).({r2})") == comp
    # star: contains identity and R(r1), and is transitive
    S = R(f"({r1})*")
    assert {(v, v) for v in range(n)} <= S and A <= S
    assert {(x, z) for (x, y) in S for (y2, z) in S if y == y2} <= S
    # plus contains R(r1)
    assert A <= R(f"({r1})+")
    # reverse: R_G(rho) = R_{G^T}(rev rho)^T
    gT = oracle.Graph(n, L, dst, src, lab)
    rev = _rev(algebra.parse(r1))
    assert {(y, x) for (x, y) in as_set(oracle.rpq(gT, rev).rows)} == A
    # vertex relabeling
    perm = np.random.Generator(np.random.PCG64(case)).permutation(n).astype(np.uint32)
    gp = oracle.Graph(n, L, perm[src], perm[dst], lab)
    assert as_set(oracle.rpq(gp, r1).rows) == {(int(perm[x]), int(perm[y])) for (x, y) in A}
    # single-source = restriction of all-pairs
    for s in (0, 7, 19):
        assert as_set(oracle.rpq(g, r1, sources=[s]).rows) == {p for p in A if p[0] == s}


@pytest.mark.parametrize("case", range(20))
def test_crpq_against_brute_force(case):
    """Definition 2 by brute force over all n^3 assignments using the
    algebra relations, against the oracle's nested-loop evaluation."""
    n, L = 9 + case % 5, 3
    src, dst, lab = synth.random_graph(n, 3 * n, L, seed=900 + case)
    vl = synth.vertex_labels(n, 2, seed=950 + case)
    g = oracle.Graph(n, L, src, dst, lab, vl)
    atoms = [(0, synth.random_regex(960 + case, L, 2), 1),
             (0, synth.random_regex(970 + case, L, 2), 2),
             (1, synth.random_regex(980 + case, L, 2), 2)]
    var_label = [-1, int(case % 2), -1]
    rel = [algebra.relation(algebra.parse(a[1]), algebra.adjacency(n, L, src, dst, lab), n) for a in atoms]
    want = []
    for f in itertools.product(range(n), repeat=3):
        if var_label[1] >= 0 and vl[f[1]] != var_label[1]:
            continue
        if all(rel[k][f[a[0]], f[a[2]]] for k, a in enumerate(atoms)):
            want.append(list(f))
    got = oracle.crpq(g, 3, atoms, var_label=var_label)
    assert got.rows.tolist() == want
    # restricting variable 0 to a sample gives the matching slice
    part = oracle.crpq(g, 3, atoms, var_label=var_label, restrict0=[1, 3])
    assert part.rows.tolist() == [t for t in want if t[0] in (1, 3)]


def test_pair_digest_is_order_independent():
    rows = np.array([[1, 2], [3, 4], [0, 9]], dtype=np.uint32)
    d1 = oracle.pair_digest(rows)
    d2 = oracle.pair_digest(rows[::-1].copy())
    assert d1 == d2 and d1[0] == 3
    assert oracle.pair_digest(np.zeros((0, 2), np.uint32)) == (0, 0, 0)


def test_label_names_with_groups():
    names = ["knows", "likes"]
    g = oracle.Graph(3, 2, np.array([0, 1], np.uint32), np.array([1, 2], np.uint32), np.array([0, 1], np.uint16))
    assert as_set(oracle.rpq(g, "knows(likes)*", names=names).rows) == {(0, 1), (0, 2)}
    assert as_set(oracle.rpq(g, "(knows|likes)+", names=names).rows) == {(0, 1), (0, 2), (1, 2)}
