"""run_rpq_static, the entry point that allocates no device memory.

It exists for callers that cannot allocate GPU memory when they query (an
application whose own pool owns the device memory, a latency-critical loop
that must not take an allocation's device-wide synchronization, code hosted
inside a runtime that forbids allocating).  Its scratch is a 64 MiB array the
library reserves per device.  This file runs last so that a failure here does
not hide the other tests; it passes on its own as well as after them.

Check: two calls in a row through the C ABI give exactly the rows of run_rpq +
fetch_pairs (bit-exact: the path is integer only)."""

import numpy as np
import pytest

from paper_2602_20748_gb300 import synth

pytestmark = pytest.mark.gpu

rpq = pytest.importorskip("paper_2602_20748_gb300.rpq")
torch = pytest.importorskip("torch")


def test_static_entry_point_matches_run_rpq():
    ctx = rpq.Context(device=0)
    src, dst, lab = synth.er_graph(1000, 5000, 4, seed=synth.BASE_SEED)
    g = rpq.load_graph(ctx, 1000, 4, src, dst, lab)
    max_rows = 200_000
    out = torch.zeros(2 * max_rows, dtype=torch.int32, device="cuda:0")
    calls = [("a.b.c*", np.array([5, 999, 17, 17, 0, 512], np.uint32)),
             ("(a|b)+.c", np.arange(300, 364, dtype=np.uint32))]
    for regex, sources in calls:
        q = rpq.compile_rpq(ctx, regex)
        n = rpq.run_rpq_static(ctx, g, q, sources, out.data_ptr(), max_rows)
        torch.cuda.synchronize()
        got = out[: 2 * n].cpu().numpy().view(np.uint32).reshape(n, 2)
        want = rpq.fetch_pairs(rpq.run_rpq(ctx, g, q, sources))
        assert n > 0
        assert np.array_equal(got, want), regex
    # a result larger than the buffer is refused with its row count
    q = rpq.compile_rpq(ctx, "(a|b|c|d)*")
    with pytest.raises(rpq.RPQError) as e:
        rpq.run_rpq_static(ctx, g, q, np.arange(64, dtype=np.uint32), out.data_ptr(), 10)
    assert e.value.code == rpq.RPQ_ERR_OUT_OF_BUDGET
