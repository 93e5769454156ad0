"""The standard, event-based executor (fresh events and waiter lists built
at every run) gives the same results as the compiled executor and the
oracle: order-sensitive CHECK state and outputs, COUNTER state, SPIN
outputs, on repeated runs."""
import numpy as np
import pytest

import oracle
from paper_2508_16522_gb300 import grt
from paper_2508_16522_gb300 import tracegen as tg

from gpu_helpers import gpu_graph, random_traces_small

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k", range(6))
def test_event_executor_check_body_equals_oracle(k):
    tr = random_traces_small(count=6, seed0=50)[k]
    g = gpu_graph(tr, body=grt.RT_BODY_CHECK, tile=(8, 8) if tr.ndim == 2 else (64, 1))
    g.analyze()
    st = out = None
    for run in range(2):
        ms = g.execute_events()
        assert ms > 0
        st, out = oracle.run_bodies(tr, oracle.oracle.BODY_CHECK, state=st)
        assert np.array_equal(g.state.cpu().numpy(), st), (tr.name, run)
        assert np.array_equal(g.out.cpu().numpy(), out), (tr.name, run)
    g.close()


def test_event_executor_counter_and_spin():
    tr = tg.stencil_1d(16, 60, 256)
    g = gpu_graph(tr, body=grt.RT_BODY_COUNTER, tile=(256, 1), state_elems=16)
    g.analyze()
    g.execute_events()
    g.execute_events()
    assert g.state.cpu().tolist() == [120] * 16
    g.close()
    tr = tg.taskbench(128, 50, "random", seed=4)
    g = gpu_graph(tr, body=grt.RT_BODY_SPIN, spin_iters=17)
    g.analyze()
    g.execute_events()
    want = np.array([oracle.spin(j, 17) for j in range(tr.n)], np.uint32).view(np.int32)
    assert np.array_equal(g.out.cpu().numpy(), want)
    # the compiled executor on the same graph agrees
    g.out.zero_()
    g.execute()
    g.sync()
    assert np.array_equal(g.out.cpu().numpy(), want)
    g.close()


def test_event_executor_full_size_graph_runs_every_task():
    tr = tg.taskbench(1024, 1000, "stencil", seed=0)
    g = gpu_graph(tr, body=grt.RT_BODY_SPIN, spin_iters=3)
    g.analyze()
    g.execute_events()
    want = np.array([oracle.spin(j, 3) for j in range(tr.n)], np.uint32).view(np.int32)
    assert np.array_equal(g.out.cpu().numpy(), want)
    g.close()
