"""Stitched replay (rt_execute_stitched): R replays of a trace T in one launch,
joined by the edges between two copies of T instead of a barrier.

Checked against the oracle's analysis of T issued R times in a row: every
edge of that DAG orders its tasks' tickets; CHECK bodies leave the state and
outputs of R sequential runs of T; SPIN and COUNTER bodies run every (replay,
task) once. Invalid inputs are refused on the host."""
import numpy as np
import pytest

import oracle
from paper_2508_16522_gb300 import grt
from paper_2508_16522_gb300 import tracegen as tg

from gpu_helpers import assert_csr_equal, ensure_built, random_traces_small

pytestmark = pytest.mark.gpu


def stitched_graph(T, R, body=grt.RT_BODY_EMPTY, spin_iters=3, flags=grt.RT_GRAPH_TICKETS, tile=(0, 0),
                   second=None):
    import torch
    ensure_built()
    T2 = tg.concat([T, second if second is not None else T])
    state = out = None
    if body == grt.RT_BODY_CHECK:
        state = torch.zeros(max(T.n_cells, 1), dtype=torch.int32, device="cuda")
    elif body == grt.RT_BODY_COUNTER:
        state = torch.zeros(int(T.body_arg.max()) + 1, dtype=torch.int32, device="cuda")
    if body in (grt.RT_BODY_CHECK, grt.RT_BODY_SPIN):
        out = torch.zeros(max(R * T.n, 2 * T.n, 1), dtype=torch.int32, device="cuda")
    g = grt.Graph(T.ndim, T.dom_lo, T.dom_hi, body=body, spin_iters=spin_iters, state=state, out=out, tile=tile,
                  flags=flags)
    g.launch_trace(T2)
    g.analyze()
    return g, T2


def check_order(g, T, R):
    n = T.n
    tk = g.stitched_tickets(R).reshape(R * n, 2)
    assert (tk >= 0).all() and len(np.unique(tk)) == 2 * R * n, "every (replay, task) ran once"
    assert (tk[:, 0] < tk[:, 1]).all()
    src, dst = oracle.analyze(tg.concat([T] * R))
    assert (tk[src, 1] < tk[dst, 0]).all(), "an edge of the replayed trace ran out of order"
    return len(src)


def small_cases():
    out = random_traces_small(count=6, seed0=70)
    out += [tg.taskbench(32, 12, p, seed=2) for p in tg.PATTERNS]
    out += [tg.taskbench(16, 8, "random", seed=3, encode="explicit"), tg.fig6_fixture(), tg.stencil_1d(8, 20, 64)]
    return out


@pytest.mark.parametrize("k", range(12))
def test_stitched_order_follows_the_replayed_dag(k):
    T = small_cases()[k]
    R = 6
    g, T2 = stitched_graph(T, R, tile=(8, 8) if T.ndim == 2 else (64, 1))
    assert_csr_equal(g, T2)
    ms = g.execute_stitched(R)
    assert ms > 0
    check_order(g, T, R)
    # again on the same graph: counters and ring start afresh
    g.execute_stitched(3)
    check_order(g, T, 3)
    g.close()


@pytest.mark.parametrize("k", range(4))
def test_stitched_check_body_equals_sequential_replays(k):
    T = random_traces_small(count=4, seed0=90)[k]
    R = 5
    g, _ = stitched_graph(T, R, body=grt.RT_BODY_CHECK, flags=0, tile=(8, 8) if T.ndim == 2 else (64, 1))
    g.execute_stitched(R)
    st, outs = None, []
    for r in range(R):
        st, out = oracle.run_bodies(T, oracle.oracle.BODY_CHECK, state=st)
        outs.append(out[:T.n].copy())
    assert np.array_equal(g.state.cpu().numpy(), st)
    assert np.array_equal(g.out.cpu().numpy()[:R * T.n], np.concatenate(outs))
    g.close()


def test_stitched_spin_and_counter_bodies():
    T = tg.taskbench(128, 40, "butterfly", seed=1)
    R = 7
    g, _ = stitched_graph(T, R, body=grt.RT_BODY_SPIN, spin_iters=11, flags=0)
    g.execute_stitched(R)
    want = np.array([oracle.spin(j, 11) for j in range(T.n)], np.uint32).view(np.int32)
    assert np.array_equal(g.out.cpu().numpy()[:R * T.n], np.tile(want, R))
    g.close()
    T = tg.stencil_1d(16, 60, 256)
    g, _ = stitched_graph(T, 4, body=grt.RT_BODY_COUNTER, flags=0, tile=(256, 1))
    g.execute_stitched(4)
    assert g.state.cpu().tolist() == [240] * 16
    g.close()


def test_stitched_full_size_stencil_runs_every_task():
    T = tg.taskbench(1024, 100, "stencil", seed=0)
    R = 20
    g, _ = stitched_graph(T, R, body=grt.RT_BODY_SPIN, spin_iters=3, flags=grt.RT_GRAPH_TICKETS)
    g.execute_stitched(R)
    want = np.array([oracle.spin(j, 3) for j in range(T.n)], np.uint32).view(np.int32)
    assert np.array_equal(g.out.cpu().numpy()[:R * T.n], np.tile(want, R))
    tk = g.stitched_tickets(R).reshape(R * T.n, 2)
    # the replays overlap: replay 1's first task starts before replay 0's last one ends
    assert tk[T.n : 2 * T.n, 0].min() < tk[: T.n, 1].max()
    g.close()


def test_stitched_refuses_invalid_input():
    T = tg.taskbench(16, 6, "stencil", seed=0)
    g, _ = stitched_graph(T, 2)
    for bad in (0, -1):
        with pytest.raises(grt.GrtError) as e:
            g.execute_stitched(bad)
        assert e.value.status == grt.RT_ERR_INVALID
    g.close()
    # halves that differ
    U = tg.taskbench(16, 6, "random", seed=5)
    g, _ = stitched_graph(T, 2, second=U)
    with pytest.raises(grt.GrtError) as e:
        g.execute_stitched(2)
    assert e.value.status == grt.RT_ERR_INVALID
    g.close()
    # an odd task count cannot hold two copies
    V = tg.taskbench(15, 1, "stencil", seed=0)
    g = grt.Graph(V.ndim, V.dom_lo, V.dom_hi)
    g.launch_trace(V)
    g.analyze()
    with pytest.raises(grt.GrtError) as e:
        g.execute_stitched(2)
    assert e.value.status == grt.RT_ERR_INVALID
    g.close()
    # SPIN needs out for every (replay, task)
    g, _ = stitched_graph(T, 2, body=grt.RT_BODY_SPIN, flags=0)
    with pytest.raises(grt.GrtError) as e:
        g.execute_stitched(40)
    assert e.value.status == grt.RT_ERR_INVALID
    g.close()
