"""Streamed materialization (rpq_stream_*) through the C ABI: the streamed
rows equal run_rpq_range's materialized rows and the CPU oracle's, block
metadata is consistent, totals (rows, digest, product edges) match, and a
source's row that spans two pinned slots is split correctly."""

import numpy as np
import pytest

import oracle
from paper_2602_20748_gb300 import synth

pytestmark = pytest.mark.gpu

rpq = pytest.importorskip("paper_2602_20748_gb300.rpq")


@pytest.fixture(scope="module")
def ctx():
    return rpq.Context(device=0)


def streamed(ctx, g, q, lo, hi, flags=0):
    st = rpq.Stream(ctx, g, q, lo, hi, flags)
    blocks = []
    while (b := st.next_block()) is not None:
        src, off, dst = (x.copy() for x in b)
        assert len(off) == len(src) + 1 and off[0] == 0 and off[-1] == len(dst)
        assert np.all(np.diff(off) > 0)  # only sources with rows in the block
        assert np.all(np.diff(src.astype(np.int64)) > 0)
        blocks.append((src, off, dst))
    info = st.info()
    st.close()
    rows = [np.stack([np.repeat(s, np.diff(o).astype(np.int64)), d], axis=1) for s, o, d in blocks]
    rows = np.concatenate(rows).astype(np.uint32) if rows else np.zeros((0, 2), dtype=np.uint32)
    return rows, info, blocks


@pytest.mark.parametrize("regex", ["a*", "a.b*.c", "(a|b)+.c", "(a.b)*", "d"])
def test_stream_equals_range_and_oracle(ctx, regex):
    n = 12000
    src, dst, lab = synth.rmat_graph(14, 6 * n, 4, 1.2, seed=71)
    src %= n
    dst %= n
    g = rpq.load_graph(ctx, n, 4, src, dst, lab)
    q = rpq.compile_rpq(ctx, regex)
    lo, hi = 1000, 10500  # three launches, the last one ragged
    rows, info, _ = streamed(ctx, g, q, lo, hi)
    r = rpq.run_rpq_range(ctx, g, q, lo, hi, rpq.RPQ_MATERIALIZE)
    want = rpq.fetch_pairs(r)
    c, _, hs, hx = rpq.result_info(r)
    w = rpq.result_stats(r)["product_edges"]
    r.free()
    assert np.array_equal(rows, want)
    assert info[0] == c and info[1] == hs and info[2] == hx and info[3]["product_edges"] == w
    # the oracle on a slice of the range
    og = oracle.Graph(n, 4, src, dst, lab)
    sl = np.arange(lo, lo + 300, dtype=np.uint32)
    o = oracle.rpq(og, regex, sources=sl)
    assert np.array_equal(rows[rows[:, 0] < lo + 300], o.rows)


def test_stream_reverse_and_empty(ctx):
    n = 5000
    src, dst, lab = synth.rmat_graph(13, 5 * n, 3, 1.2, seed=72)
    src %= n
    dst %= n
    g = rpq.load_graph(ctx, n, 3, src, dst, lab)
    q = rpq.compile_rpq(ctx, "a.b*")
    rows, info, blocks = streamed(ctx, g, q, 0, n, rpq.RPQ_REVERSE)
    r = rpq.run_rpq_range(ctx, g, q, 0, n, rpq.RPQ_MATERIALIZE | rpq.RPQ_REVERSE)
    assert np.array_equal(rows, rpq.fetch_pairs(r))
    r.free()
    rows, info, blocks = streamed(ctx, g, q, 17, 17)
    assert len(rows) == 0 and info[0] == 0 and not blocks
    with pytest.raises(rpq.RPQError):
        rpq.Stream(ctx, g, q, 0, n + 1)
    with pytest.raises(rpq.RPQError):
        rpq.Stream(ctx, g, q, 0, n, rpq.RPQ_COUNT_ONLY)


def test_stream_row_split_across_slots(ctx):
    # a* on a strongly connected graph: every source reaches every vertex, so
    # one launch holds 4,096 x n rows, more than a pinned slot (2^26), and the
    # row that crosses the slot boundary is split over two blocks
    n = 20000
    rng = np.random.Generator(np.random.PCG64(73))
    src = np.concatenate([np.arange(n), rng.integers(0, n, 3 * n)]).astype(np.uint32)
    dst = np.concatenate([(np.arange(n) + 1) % n, rng.integers(0, n, 3 * n)]).astype(np.uint32)
    lab = np.zeros(len(src), dtype=np.uint16)
    g = rpq.load_graph(ctx, n, 1, src, dst, lab)
    q = rpq.compile_rpq(ctx, "a*")
    rows, info, blocks = streamed(ctx, g, q, 0, 4096)
    assert info[0] == 4096 * n and len(rows) == 4096 * n
    assert len(blocks) == 2
    cut = (1 << 26) // n  # source whose row crosses the boundary
    assert blocks[0][0][-1] == cut and blocks[1][0][0] == cut
    assert np.array_equal(rows[:, 0], np.repeat(np.arange(4096, dtype=np.uint32), n))
    assert np.array_equal(rows[:, 1], np.tile(np.arange(n, dtype=np.uint32), 4096))


def test_stream_multi_query_equals_single(ctx):
    """rpq_stream_open_multi: the blocks of each query, in order, give exactly
    that query's single-query stream rows; totals are the sums."""
    n = 9000
    src, dst, lab = synth.rmat_graph(14, 6 * n, 4, 1.2, seed=73)
    src %= n
    dst %= n
    g = rpq.load_graph(ctx, n, 4, src, dst, lab)
    regexes = ["a*", "d", "(a|b)+.c", "a.b*.c"]
    qs = [rpq.compile_rpq(ctx, r) for r in regexes]
    lo, hi = 300, 8900  # three launches per query, the last one ragged
    st = rpq.Stream(ctx, g, qs, lo, hi)
    per_q = [[] for _ in qs]
    last = 0
    while (b := st.next_block()) is not None:
        s_, o_, d_ = (x.copy() for x in b)
        assert st.block_query >= last  # queries arrive one after another
        last = st.block_query
        per_q[st.block_query].append(np.stack([np.repeat(s_, np.diff(o_).astype(np.int64)), d_], axis=1))
    rows_m, hs_m, hx_m, stats_m = st.info()
    st.close()
    tot, hs, hx, w = 0, 0, 0, 0
    for i, q in enumerate(qs):
        got = np.concatenate(per_q[i]).astype(np.uint32) if per_q[i] else np.zeros((0, 2), dtype=np.uint32)
        want, info, _ = streamed(ctx, g, q, lo, hi)
        assert np.array_equal(got, want), regexes[i]
        tot += info[0]
        hs = (hs + info[1]) % (1 << 64)
        hx ^= info[2]
        w += info[3]["product_edges"]
    assert rows_m == tot and hs_m == hs and hx_m == hx and stats_m["product_edges"] == w
    with pytest.raises(rpq.RPQError):
        rpq.Stream(ctx, g, [], lo, hi)
