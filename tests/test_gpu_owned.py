"""The owned-chunk executor policy (RT_EXEC_OWNED): every warp owns fixed
chunks of consecutive tasks (32 / L of them, L lanes per task) and polls their
countdowns. Results must be those of the ring policy and of the oracle:
order-sensitive CHECK and COUNTER bodies equal sequential execution, replays
equal repeated runs, tickets order every edge, a held task ends the run with a
bounded wait, and launch shapes down to one warp (which owns every chunk) and
every group size give the same results -- also for out-degrees on both sides
of what the trigger records hold inline (5, and 13 with the extension
record)."""
import numpy as np
import pytest

import oracle
from paper_2508_16522_gb300 import grt
from paper_2508_16522_gb300 import tracegen as tg

from gpu_helpers import gpu_graph, oracle_csr

pytestmark = pytest.mark.gpu

# (blocks, warps, lanes per task); 0 = default
SHAPES = [(0, 0, 0), (1, 1, 1), (3, 2, 2), (152, 4, 4), (7, 1, 4), (64, 1, 2)]


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
        g.exec_config(shape[0], shape[1], shape[2])
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


@pytest.mark.parametrize("shape", [(0, 0, 0), (1, 1, 1), (304, 2, 2), (128, 1, 4)])
def test_tickets_order_every_edge(shape):
    for tr in [tg.taskbench(1024, 200, "random"), tg.taskbench(1024, 200, "stencil"),
               tg.random_rects(grid=(64, 64), n=3000, side=(2, 24), seed=5)]:
        g = gpu_graph(tr, flags=grt.RT_GRAPH_TICKETS)
        g.analyze()
        g.exec_policy(grt.RT_EXEC_OWNED)
        g.exec_config(shape[0], shape[1], shape[2])
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


def hub_trace(ks=(4, 5, 6, 12, 13, 14, 40)):
    """1-D hubs: for each k, a task writes k cells, k tasks read one cell each
    (the writer's out-degree is k), and a task writes the k cells again (its
    in-degree is k)."""
    lo, hi, priv = [], [], []
    base = 0
    for k in ks:
        lo.append(base); hi.append(base + k - 1); priv.append(tg.WRITE)
        for i in range(k):
            lo.append(base + i); hi.append(base + i); priv.append(tg.READ)
        lo.append(base); hi.append(base + k - 1); priv.append(tg.WRITE)
        base += k
    n = len(priv)
    return tg.Trace(ndim=1, dom_lo=np.array([0], np.int64), dom_hi=np.array([base - 1], np.int64),
                    req_off=np.arange(n + 1, dtype=np.int32), lo=np.array(lo, np.int64).reshape(n, 1),
                    hi=np.array(hi, np.int64).reshape(n, 1), priv=np.array(priv, np.uint8), name="hubs")


@pytest.mark.parametrize("group", [1, 2, 4])
def test_out_degrees_around_the_inline_record(group):
    for tr in (hub_trace(), hub_trace((2, 3, 5)), tg.taskbench(1024, 60, "random", seed=9)):
        rp_o, col_o, _ = oracle_csr(tr)
        deg = np.diff(rp_o)
        for blocks in (1, 7, 64):
            g = gpu_graph(tr, body=grt.RT_BODY_CHECK, flags=grt.RT_GRAPH_TICKETS,
                          tile=(64, 1) if tr.ndim == 1 else (16, 16))
            g.analyze()
            g.exec_policy(grt.RT_EXEC_OWNED)
            g.exec_config(blocks, 1, group)
            g.execute()
            g.sync()
            st, out = oracle.run_bodies(tr, oracle.BODY_CHECK)
            assert np.array_equal(g.state.cpu().numpy(), st), (tr.name, blocks)
            assert np.array_equal(g.out.cpu().numpy(), out), (tr.name, blocks)
            t = g.tickets()
            src = np.repeat(np.arange(tr.n), deg)
            assert (t[src, 1] < t[col_o, 0]).all(), (tr.name, blocks)
            c = g.stats()["exec_counters"]
            assert c["tasks"] == tr.n and c["edges"] == len(col_o), (tr.name, blocks, c)
            g.close()
        if tr.name == "hubs" and deg.max() > 13:
            assert {5, 6, 13, 14} <= set(deg.tolist())


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
