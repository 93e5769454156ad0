"""Tasks as whole kernels (Section 4.3): lifted, async-edge and CUDA-graph
runs of the same DAG. Each task kernel writes 1 + the largest output of its
predecessors, so the outputs equal the tasks' depths only if every
predecessor finished first."""
import numpy as np
import pytest

import oracle
from paper_2508_16522_gb300 import grt
from paper_2508_16522_gb300 import tracegen as tg

from gpu_helpers import gpu_graph, oracle_csr

pytestmark = pytest.mark.gpu


def depths(tr):
    rp, col, _ = oracle_csr(tr)
    order = oracle.topo_order(tr.n, rp, col)
    d = np.ones(tr.n, np.int64)
    for v in order:
        for s in col[rp[v]:rp[v + 1]]:
            d[s] = max(d[s], d[v] + 1)
    return d


@pytest.mark.parametrize("tr", [tg.taskbench(8, 60, "stencil", seed=1), tg.taskbench(16, 40, "random", seed=2),
                                tg.random_rects(grid=(40, 30), n=500, rects=(1, 3), side=(1, 9), seed=3)],
                         ids=["stencil", "random", "rects"])
def test_every_mode_respects_the_edges(tr):
    want = depths(tr)
    g = gpu_graph(tr, body=grt.RT_BODY_SPIN, spin_iters=0)
    g.analyze()
    for mode in ("lifted", "async", "graph", "graph"):  # the graph is instantiated once, then relaunched
        ms = g.execute_kernels(mode, iters=64, threads=64)
        assert ms > 0
        assert np.array_equal(g.out.cpu().numpy().astype(np.int64), want), (tr.name, mode)
    g.close()


def test_kernel_mode_arguments_are_checked():
    tr = tg.taskbench(8, 4, "stencil", seed=1)
    g = gpu_graph(tr)  # EMPTY body: no out buffer
    g.analyze()
    with pytest.raises(grt.GrtError) as e:
        g.execute_kernels("async")
    assert e.value.status == grt.RT_ERR_INVALID
    g.close()
