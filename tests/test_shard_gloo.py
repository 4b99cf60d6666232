"""Multi-rank path on CPU: two gloo ranks split an all-pairs job by batches of
start vertices (paper_2602_20748_gb300.shard), each evaluates its batches
with the CPU oracle, and the combined summary (rows, digest, work) equals the
single-process result over all start vertices; the ranks' batches are
disjoint and cover the job."""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
from paper_2602_20748_gb300 import shard, synth  # noqa: E402

N, M, L = 512, 2600, 3
B = 64  # start vertices per batch
REGEX = "a.b*"


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _summary(g, batches):
    rows = np.zeros((0, 2), dtype=np.uint32)
    work = 0
    for b in batches:
        r = oracle.rpq(g, REGEX, sources=np.arange(b * B, (b + 1) * B, dtype=np.uint32))
        rows = np.concatenate([rows, r.rows])
        work += r.W
    cnt, s, x = oracle.pair_digest(rows)
    return {"rows": cnt, "digest_sum": s, "digest_xor": x, "work": work, "ms": 1.0}


def _rank(rank, world, port, steps, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        src, dst, lab = synth.er_graph(N, M, L, seed=synth.BASE_SEED + 9)
        g = oracle.Graph(N, L, src, dst, lab)
        mine = shard.rank_batches(N // B, 0, steps, world, rank)
        allb = [None] * world
        dist.all_gather_object(allb, mine)
        tot = shard.gather_combine(dist, _summary(g, mine))
        if rank == 0:
            out.put((allb, tot))
    finally:
        dist.destroy_process_group()


def test_two_ranks_partition_and_combine():
    world, steps = 2, (N // B) // 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    allb, tot = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    flat = sorted(b for bs in allb for b in bs)
    assert flat == list(range(N // B))  # disjoint and complete
    src, dst, lab = synth.er_graph(N, M, L, seed=synth.BASE_SEED + 9)
    whole = oracle.rpq(oracle.Graph(N, L, src, dst, lab), REGEX)
    cnt, s, x = oracle.pair_digest(whole.rows)
    assert (tot["rows"], tot["digest_sum"], tot["digest_xor"], tot["work"]) == (cnt, s, x, whole.W)


def test_rank_batches_and_combine_host_logic():
    assert shard.rank_batches(8, 0, 4, 2, 0) == [0, 2, 4, 6]
    assert shard.rank_batches(8, 0, 4, 2, 1) == [1, 3, 5, 7]
    assert shard.rank_batches(5, 3, 2, 1, 0) == [3, 4]
    with pytest.raises(ValueError):
        shard.rank_batches(8, 0, 1, 2, 2)
    c = shard.combine([{"rows": 2, "digest_sum": (1 << 64) - 1, "digest_xor": 5, "work": 7, "ms": 3.0},
                       {"rows": 1, "digest_sum": 2, "digest_xor": 3, "work": 1, "ms": 4.5}])
    assert c == {"rows": 3, "digest_sum": 1, "digest_xor": 6, "work": 8, "ms": 4.5}
