"""The FMA body (Task Bench's floating-point loop: dependent binary32 fused
multiply-adds on one lane) through every executor: its per-task result bits
equal the oracle's, which is pinned to exact rational rounding on the CPU."""
import numpy as np
import pytest

import oracle
from paper_2508_16522_gb300 import grt
from paper_2508_16522_gb300 import tracegen as tg

from gpu_helpers import ensure_built, gpu_graph

pytestmark = pytest.mark.gpu

ITERS = 37


def want(n, iters=ITERS):
    return np.array([oracle.fma_bits(v, iters) for v in range(n)], np.uint32).view(np.int32)


def test_fma_compiled_replay_and_events():
    ensure_built()
    for tr in (tg.taskbench(64, 40, "random", seed=2), tg.random_rects(grid=(48, 40), n=500, side=(1, 10), seed=9)):
        g = gpu_graph(tr, body=grt.RT_BODY_FMA, spin_iters=ITERS)
        g.analyze()
        g.execute()
        g.sync()
        assert np.array_equal(g.out.cpu().numpy()[:tr.n], want(tr.n)), tr.name
        g.out.zero_()
        g.replay(3)
        g.sync()
        assert np.array_equal(g.out.cpu().numpy()[:tr.n], want(tr.n)), tr.name
        g.out.zero_()
        g.execute_events()
        assert np.array_equal(g.out.cpu().numpy()[:tr.n], want(tr.n)), tr.name
        g.close()


def test_fma_in_a_batch_and_stitched():
    ensure_built()
    traces = [tg.taskbench(32, 20 + 5 * k, "stencil", seed=k) for k in range(5)]
    graphs = []
    for tr in traces:
        g = gpu_graph(tr, body=grt.RT_BODY_FMA, spin_iters=ITERS)
        g.analyze()
        graphs.append(g)
    b = grt.Batch(graphs)
    b.execute(replays=2)
    b.sync()
    for tr, g in zip(traces, graphs):
        assert np.array_equal(g.out.cpu().numpy()[:tr.n], want(tr.n)), tr.name
    b.close()
    for g in graphs:
        g.close()
    T = tg.taskbench(64, 30, "butterfly", seed=1)
    R = 4
    two = tg.concat([T, T])
    import torch
    out = torch.zeros(R * T.n, dtype=torch.int32, device="cuda")
    g = grt.Graph(2, two.dom_lo, two.dom_hi, body=grt.RT_BODY_FMA, spin_iters=ITERS, out=out)
    g.launch_trace(two)
    g.analyze()
    g.execute_stitched(R)
    assert np.array_equal(out.cpu().numpy(), np.tile(want(T.n), R))
    g.close()
