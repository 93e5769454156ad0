"""The owned-chunk executor policy (RT_EXEC_OWNED): every warp owns fixed
chunks of 32 consecutive tasks and polls their countdowns. Results must be
those of the ring policy and of the oracle: order-sensitive CHECK and COUNTER
bodies equal sequential execution, replays equal repeated runs, tickets order
every edge, a held task ends the run with a bounded wait, and launch shapes
down to one warp (which owns every chunk) give the same results."""
import numpy as np
import pytest

import oracle
from paper_2508_16522_gb300 import grt
from paper_2508_16522_gb300 import tracegen as tg

from gpu_helpers import gpu_graph

pytestmark = pytest.mark.gpu

SHAPES = [(0, 0), (1, 1), (3, 2), (152, 4)]  # (blocks, warps); (0, 0) = default


def traces():
    return [tg.random_rects(grid=(40, 30), n=700, rects=(1, 4), side=(1, 12), seed=21),
            tg.taskbench(96, 40, "random", seed=3),
            tg.random_rects(grid=(500,), n=400, rects=(1, 3), side=(1, 60), seed=22, ndim=1)]


@pytest.mark.parametrize("shape", SHAPES)
def test_check_body_and_replays(shape):
    for tr in traces():
        g = gpu_graph(tr, body=grt.RT_BODY_CHECK, tile=(8, 8) if tr.ndim == 2 else (64, 1))
        g.analyze()
        g.exec_policy(grt.RT_EXEC_OWNED)
        g.exec_config(shape[0], shape[1])
        g.execute()
        g.sync()
        st, out = oracle.run_bodies(tr, oracle.BODY_CHECK)
        assert np.array_equal(g.state.cpu().numpy(), st), tr.name
        assert np.array_equal(g.out.cpu().numpy(), out), tr.name
        for reps in (3, 3):  # the second time from the cached CUDA graph
            g.replay(reps)
            g.sync()
            for _ in range(reps):
                st, out = oracle.run_bodies(tr, oracle.BODY_CHECK, state=st)
            assert np.array_equal(g.state.cpu().numpy(), st), tr.name
            assert np.array_equal(g.out.cpu().numpy(), out), tr.name
        g.close()


def test_counter_and_fma_bodies():
    tr = tg.stencil_1d()
    g = gpu_graph(tr, body=grt.RT_BODY_COUNTER, state_elems=16)
    g.analyze()
    g.exec_policy(grt.RT_EXEC_OWNED)
    g.replay(4)
    g.sync()
    assert g.state.cpu().numpy().tolist() == [400] * 16
    g.close()
    tr = tg.taskbench(256, 30, "butterfly")
    g = gpu_graph(tr, body=grt.RT_BODY_FMA, spin_iters=33)
    g.analyze()
    g.exec_policy(grt.RT_EXEC_OWNED)
    g.execute()
    g.sync()
    want = np.array([oracle.fma_bits(v, 33) for v in range(tr.n)], np.uint32).view(np.int32)
    assert np.array_equal(g.out.cpu().numpy(), want)
    g.close()


@pytest.mark.parametrize("shape", [(0, 0), (1, 1), (304, 2)])
def test_tickets_order_every_edge(shape):
    for tr in [tg.taskbench(1024, 200, "random"), tg.taskbench(1024, 200, "stencil"),
               tg.random_rects(grid=(64, 64), n=3000, side=(2, 24), seed=5)]:
        g = gpu_graph(tr, flags=grt.RT_GRAPH_TICKETS)
        g.analyze()
        g.exec_policy(grt.RT_EXEC_OWNED)
        g.exec_config(shape[0], shape[1])
        g.execute()
        g.sync()
        t = g.tickets()
        rp, col, _ = g.csr()
        src = np.repeat(np.arange(tr.n), np.diff(rp))
        assert (t[src, 1] < t[col, 0]).all(), "a task started before one of its predecessors finished"
        assert sorted(np.concatenate([t[:, 0], t[:, 1]]).tolist()) == list(range(2 * tr.n))
        st = g.stats()
        assert st["exec_counters"]["tasks"] == tr.n and st["exec_counters"]["edges"] == len(col)
        g.close()


def test_bounded_wait_timeout_and_recovery():
    tr = tg.taskbench(64, 20, "stencil")
    g = gpu_graph(tr, body=grt.RT_BODY_SPIN, spin_iters=4, timeout_ns=300_000_000)
    g.analyze()
    g.exec_policy(grt.RT_EXEC_OWNED)
    g.hold_task(64 * 10 + 5)  # never becomes ready
    g.execute()
    with pytest.raises(grt.GrtError) as e:
        g.sync()
    assert e.value.status == grt.RT_ERR_TIMEOUT
    g.execute()
    g.sync()
    want = np.array([oracle.spin(j, 4) for j in range(tr.n)], np.uint32).view(np.int32)
    assert np.array_equal(g.out.cpu().numpy(), want)
    # a held task in a replay: the warps waiting at the run barrier give up too
    g.hold_task(64 * 3 + 1)
    g.replay(3)
    with pytest.raises(grt.GrtError) as e:
        g.sync()
    assert e.value.status == grt.RT_ERR_TIMEOUT
    g.replay(2)
    g.sync()
    g.close()


def test_policy_switches_back_and_forth():
    tr = tg.random_rects(grid=(48, 40), n=900, side=(1, 10), seed=8)
    g = gpu_graph(tr, body=grt.RT_BODY_CHECK, tile=(16, 16))
    g.analyze()
    st = None
    for pol in (grt.RT_EXEC_OWNED, grt.RT_EXEC_RING, grt.RT_EXEC_OWNED):
        g.exec_policy(pol)
        g.replay(2)
        g.sync()
        for _ in range(2):
            st, out = oracle.run_bodies(tr, oracle.BODY_CHECK, state=st)
        assert np.array_equal(g.state.cpu().numpy(), st)
        assert np.array_equal(g.out.cpu().numpy(), out)
    with pytest.raises(grt.GrtError):
        g.exec_policy(7)
    g.close()
