"""run_rpq_static, the entry point that allocates no device memory.

It exists for callers that cannot allocate GPU memory when they query (an
application whose own pool owns the device memory, a latency-critical loop
that must not take an allocation's device-wide synchronization, code hosted
inside a runtime that forbids allocating).  Its scratch is a 64 MiB array the
library reserves per device when the first context is created.  This file
runs last so that a failure here does not hide the other tests; it passes on
its own as well as after them.

Checks, all through the C ABI and bit-exact (the path is integer only):
two calls in a row give the rows of run_rpq + fetch_pairs and of the CPU
oracle; hub vertices whose rows are scanned in place (this entry point keeps
no chunk lists and no spill records); a language containing the empty word;
a label the graph lacks; the size and argument refusals; free device memory
unchanged by a call; and calls on a device whose memory is otherwise full."""

import numpy as np
import pytest

import oracle
from paper_2602_20748_gb300 import synth

pytestmark = pytest.mark.gpu

rpq = pytest.importorskip("paper_2602_20748_gb300.rpq")
torch = pytest.importorskip("torch")

MAX_ROWS = 400_000


@pytest.fixture(scope="module")
def ctx():
    return rpq.Context(device=0)


@pytest.fixture(scope="module")
def out():
    return torch.zeros(2 * MAX_ROWS, dtype=torch.int32, device="cuda:0")


def _static_rows(ctx, g, q, sources, out):
    n = rpq.run_rpq_static(ctx, g, q, sources, out.data_ptr(), MAX_ROWS)
    torch.cuda.synchronize()
    return out[: 2 * n].cpu().numpy().view(np.uint32).reshape(n, 2)


def _hub_graph():
    """ER background plus hubs: vertex 7 has 3,000 out-edges and vertex 11
    3,000 in-edges on label a (rows far above the in-place thresholds of 128
    and 1,024 edges), vertex 13 both on label b."""
    n = 4000
    s, d, l = synth.er_graph(n, 12000, 3, seed=synth.BASE_SEED + 77)
    rng = np.random.Generator(np.random.PCG64(5))
    hs = [np.full(3000, 7), rng.integers(0, n, 3000), np.full(1500, 13), rng.integers(0, n, 1500)]
    hd = [rng.integers(0, n, 3000), np.full(3000, 11), rng.integers(0, n, 1500), np.full(1500, 13)]
    hl = [np.zeros(3000), np.zeros(3000), np.ones(1500), np.ones(1500)]
    src = np.concatenate([s] + hs).astype(np.uint32)
    dst = np.concatenate([d] + hd).astype(np.uint32)
    lab = np.concatenate([l] + hl).astype(np.uint16)
    return n, src, dst, lab


def test_static_entry_point_matches_run_rpq_and_oracle(ctx, out):
    src, dst, lab = synth.er_graph(1000, 5000, 4, seed=synth.BASE_SEED)
    g = rpq.load_graph(ctx, 1000, 4, src, dst, lab)
    og = oracle.Graph(1000, 4, src, dst, lab)
    calls = [("a.b.c*", np.array([5, 999, 17, 17, 0, 512], np.uint32)),
             ("(a|b)+.c", np.arange(300, 364, dtype=np.uint32))]
    for regex, sources in calls:
        q = rpq.compile_rpq(ctx, regex)
        got = _static_rows(ctx, g, q, sources, out)
        want = rpq.fetch_pairs(rpq.run_rpq(ctx, g, q, sources))
        assert len(got) > 0
        assert np.array_equal(got, want), regex
        assert np.array_equal(got, oracle.rpq(og, regex, sources=np.unique(sources)).rows), regex
    # a result larger than the buffer is refused with its row count
    q = rpq.compile_rpq(ctx, "(a|b|c|d)*")
    with pytest.raises(rpq.RPQError) as e:
        rpq.run_rpq_static(ctx, g, q, np.arange(64, dtype=np.uint32), out.data_ptr(), 10)
    assert e.value.code == rpq.RPQ_ERR_OUT_OF_BUDGET


@pytest.mark.parametrize("regex", ["a*", "a+.b", "b.a*", "(a|b)*.c", "c*.b+"])
def test_static_hub_rows_in_place(ctx, out, regex):
    n, src, dst, lab = _hub_graph()
    g = rpq.load_graph(ctx, n, 3, src, dst, lab)
    og = oracle.Graph(n, 3, src, dst, lab)
    sources = np.array([7, 11, 13, 0, 1, 2, 3999], np.uint32)
    q = rpq.compile_rpq(ctx, regex)
    for flags in (0, rpq.RPQ_FORCE_PUSH, rpq.RPQ_FORCE_PULL):
        # reference rows from run_rpq in each expansion direction
        want = rpq.fetch_pairs(rpq.run_rpq(ctx, g, q, sources, flags=rpq.RPQ_MATERIALIZE | flags))
        assert np.array_equal(want, oracle.rpq(og, regex, sources=np.unique(sources)).rows)
    got = _static_rows(ctx, g, q, sources, out)
    assert np.array_equal(got, want), regex


def test_static_empty_word_and_absent_label(ctx, out):
    src, dst, lab = synth.er_graph(1000, 5000, 4, seed=synth.BASE_SEED)
    g = rpq.load_graph(ctx, 1000, 4, src, dst, lab)
    og = oracle.Graph(1000, 4, src, dst, lab)
    sources = np.arange(0, 1000, 16, dtype=np.uint32)
    # the empty word: (s, s) for every start vertex (Definition 1, paths of length 0)
    for regex in ("a*", "(a.b)*", "a?.b*"):
        q = rpq.compile_rpq(ctx, regex)
        got = _static_rows(ctx, g, q, sources, out)
        assert np.array_equal(got, oracle.rpq(og, regex, sources=sources).rows), regex
        assert all((s, s) in set(map(tuple, got.tolist())) for s in sources.tolist())
    # label z is not in the graph: no rows; z* matches only the empty word
    q = rpq.compile_rpq(ctx, "z")
    assert len(_static_rows(ctx, g, q, sources, out)) == 0
    q = rpq.compile_rpq(ctx, "z*")
    got = _static_rows(ctx, g, q, sources, out)
    assert np.array_equal(got, np.stack([sources, sources], axis=1))


def test_static_refusals(ctx, out):
    src, dst, lab = synth.er_graph(1000, 5000, 4, seed=synth.BASE_SEED)
    g = rpq.load_graph(ctx, 1000, 4, src, dst, lab)
    q = rpq.compile_rpq(ctx, "a*")
    for bad in (np.arange(65, dtype=np.uint32), np.array([1000], np.uint32), np.zeros(0, np.uint32)):
        with pytest.raises(rpq.RPQError) as e:
            rpq.run_rpq_static(ctx, g, q, bad, out.data_ptr(), MAX_ROWS)
        assert e.value.code == rpq.RPQ_ERR_INVALID_ARG
    # 2^21 vertices need about 5 * 8 bytes per (state, vertex): more than the 64 MiB array
    n = 1 << 21
    big = rpq.load_graph(ctx, n, 1, np.array([0, 1], np.uint32), np.array([1, 2], np.uint32),
                         np.zeros(2, np.uint16))
    with pytest.raises(rpq.RPQError) as e:
        rpq.run_rpq_static(ctx, big, q, np.array([0], np.uint32), out.data_ptr(), MAX_ROWS)
    assert e.value.code == rpq.RPQ_ERR_OUT_OF_BUDGET
    assert "67108864" in str(e.value)


def test_static_allocates_nothing(ctx, out):
    src, dst, lab = synth.er_graph(1000, 5000, 4, seed=synth.BASE_SEED)
    g = rpq.load_graph(ctx, 1000, 4, src, dst, lab)
    q = rpq.compile_rpq(ctx, "(a|b)+.c")
    sources = np.arange(100, 164, dtype=np.uint32)
    first = _static_rows(ctx, g, q, sources, out).copy()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(0)[0]
    second = _static_rows(ctx, g, q, sources, out).copy()
    free1 = torch.cuda.mem_get_info(0)[0]
    assert free1 >= free0
    assert np.array_equal(first, second)
    # the rest of the device taken by someone else's pool: the calls still run
    spare = 256 << 20
    hog = None
    if free1 > 2 * spare:
        hog = torch.empty(free1 - spare, dtype=torch.uint8, device="cuda:0")
    try:
        for _ in range(2):
            assert np.array_equal(_static_rows(ctx, g, q, sources, out), first)
    finally:
        del hog
        torch.cuda.empty_cache()
