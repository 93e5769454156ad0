"""Batched execution: many captured graphs in one persistent launch, each
replayed independently. Every graph's result in the batch must equal its
result alone (the oracle's sequential execution, repeated per replay)."""
import numpy as np
import pytest

import oracle
from paper_2508_16522_gb300 import grt
from paper_2508_16522_gb300 import tracegen as tg

from gpu_helpers import gpu_graph

pytestmark = pytest.mark.gpu


def _oracle_repeat(tr, body, reps, spin_iters=256, state_elems=None):
    st = np.zeros(state_elems, np.int32) if state_elems else None
    out = None
    for _ in range(reps):
        st, out = oracle.run_bodies(tr, body, state=st, spin_iters=spin_iters)
    return st, out


@pytest.mark.parametrize("replays", [1, 3])
def test_mixed_batch_equals_each_graph_alone(replays):
    traces, bodies = [], []
    for k in range(24):
        if k % 4 == 0:
            traces.append(tg.random_rects(grid=(30, 22), n=150 + 10 * k, rects=(1, 3), side=(1, 9), seed=100 + k))
            bodies.append(grt.RT_BODY_CHECK)
        elif k % 4 == 1:
            traces.append(tg.taskbench(32, 5 + k, tg.PATTERNS[k % 3], seed=k))
            bodies.append(grt.RT_BODY_SPIN)
        elif k % 4 == 2:
            traces.append(tg.stencil_1d(8, 3 + k, 64))
            bodies.append(grt.RT_BODY_COUNTER)
        else:
            traces.append(tg.taskbench(16, 9, "butterfly", encode="explicit"))
            bodies.append(grt.RT_BODY_EMPTY)
    graphs = []
    for tr, b in zip(traces, bodies):
        g = gpu_graph(tr, body=b, spin_iters=37, tile=(8, 8) if tr.ndim == 2 else (64, 1),
                      state_elems=8 if b == grt.RT_BODY_COUNTER else None)
        g.analyze()
        graphs.append(g)
    batch = grt.Batch(graphs)
    batch.execute(replays=replays)
    ms = batch.sync()
    assert ms > 0
    for tr, b, g in zip(traces, bodies, graphs):
        if b == grt.RT_BODY_CHECK:
            st, out = _oracle_repeat(tr, oracle.oracle.BODY_CHECK, replays)
            assert np.array_equal(g.state.cpu().numpy(), st), tr.name
            assert np.array_equal(g.out.cpu().numpy(), out), tr.name
        elif b == grt.RT_BODY_SPIN:
            want = np.array([oracle.spin(j, 37) for j in range(tr.n)], np.uint32).view(np.int32)
            assert np.array_equal(g.out.cpu().numpy(), want), tr.name
        elif b == grt.RT_BODY_COUNTER:
            st, _ = _oracle_repeat(tr, oracle.oracle.BODY_COUNTER, replays, state_elems=8)
            assert np.array_equal(g.state.cpu().numpy(), st), tr.name
    # the batch can run again (counters re-armed by the tasks themselves)
    batch.execute(replays=1)
    batch.sync()
    batch.close()
    for g in graphs:
        g.close()


def test_batch_with_empty_and_single_task_graphs():
    import torch
    empty = grt.Graph(2, [0, 0], [3, 3])
    empty.analyze()
    one = gpu_graph(tg._finish(2, [0, 0], [3, 3], [1], np.array([0, 0]), np.array([3, 3]),
                               np.array([1], np.uint8)), body=grt.RT_BODY_SPIN, spin_iters=5)
    one.analyze()
    big = gpu_graph(tg.taskbench(64, 30, "random"), body=grt.RT_BODY_SPIN, spin_iters=5)
    big.analyze()
    b = grt.Batch([empty, one, big])
    b.execute(replays=4)
    b.sync()
    assert one.out.cpu().tolist() == [oracle.spin(0, 5)]
    want = np.array([oracle.spin(j, 5) for j in range(64 * 30)], np.uint32).view(np.int32)
    assert np.array_equal(big.out.cpu().numpy(), want)
    b.close()
    for g in (empty, one, big):
        g.close()
    del torch


@pytest.mark.parametrize("shape", [(0, 0, 0, 0), (152, 2, 8, 8), (304, 4, 32, 64), (1, 1, 1, 0)])
def test_batch_launch_shapes_give_same_results(shape):
    gs_tr = tg.batch_graphs(60, n_range=(64, 4096), seed=3)
    graphs = []
    for tr in gs_tr:
        g = gpu_graph(tr, body=grt.RT_BODY_SPIN, spin_iters=3, tile=(8, 8))
        g.analyze()
        graphs.append(g)
    b = grt.Batch(graphs)
    blocks, warps, claim, keep = shape
    b.execute(replays=2, blocks=blocks, warps=warps, claim=claim, keep=keep)
    b.sync()
    for tr, g in zip(gs_tr, graphs):
        want = np.array([oracle.spin(j, 3) for j in range(tr.n)], np.uint32).view(np.int32)
        assert np.array_equal(g.out.cpu().numpy(), want), tr.name
    b.close()
    for g in graphs:
        g.close()
