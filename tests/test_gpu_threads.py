"""Calls on distinct graphs from distinct host threads: several graphs, each on
its own stream, ingested, analysed and executed at the same time by their own
threads, give each the oracle's CSR and the oracle's order-sensitive CHECK
results -- the same as each graph alone."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_2508_16522_gb300 import grt
from paper_2508_16522_gb300 import tracegen as tg

from gpu_helpers import assert_csr_equal, ensure_built, gpu_graph, oracle_csr

pytestmark = pytest.mark.gpu


def test_graphs_analysed_and_executed_concurrently():
    import torch
    ensure_built()
    trs = [tg.random_rects(grid=(200, 150), n=3000, rects=(1, 4), side=(1, 30), seed=41 + k) for k in range(3)]
    trs += [tg.taskbench(512, 60, p, seed=5) for p in tg.PATTERNS]
    refs = [oracle_csr(t) for t in trs]
    want = [oracle.run_bodies(t, oracle.BODY_CHECK) for t in trs]
    streams = [torch.cuda.Stream() for _ in trs]
    graphs = [gpu_graph(t, body=grt.RT_BODY_CHECK, tile=(16, 16), stream=s, defer_check=True)
              for t, s in zip(trs, streams)]

    def work(k):
        torch.cuda.set_device(0)
        g = graphs[k]
        for rep in range(3):  # analysis and execution again and again, overlapping the other threads'
            if rep:
                g.clear()
                g.state.zero_()
                torch.cuda.current_stream().synchronize()  # the zeroing before the graph's own stream
                g.launch_trace(trs[k], defer_check=True)
            g.analyze()
            g.execute()
            g.sync()
        return k

    with ThreadPoolExecutor(max_workers=len(trs)) as pool:
        assert sorted(pool.map(work, range(len(trs)))) == list(range(len(trs)))
    for g, t, ref, (st, out) in zip(graphs, trs, refs, want):
        assert_csr_equal(g, t, ref)
        assert np.array_equal(g.state.cpu().numpy(), st), t.name
        assert np.array_equal(g.out.cpu().numpy(), out), t.name
        g.close()
