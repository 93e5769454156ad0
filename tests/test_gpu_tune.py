"""The autotuner: it picks among candidate tiles and launch shapes by measuring
them on the caller's workload, answers a repeated workload from its cache, and
whatever it picks, the results stay those of the oracle."""
import numpy as np
import pytest

import oracle
from paper_2508_16522_gb300 import grt
from paper_2508_16522_gb300 import tracegen as tg

from gpu_helpers import assert_csr_equal, ensure_built, gpu_graph

pytestmark = pytest.mark.gpu


def test_tile_tuner_picks_a_candidate_and_caches_it(tmp_path):
    ensure_built()
    cache = tmp_path / "tune.txt"
    tr = tg.random_rects(grid=(300, 200), n=3000, rects=(1, 3), side=(1, 40), seed=31)
    tw, th, ms = grt.rt_tune_tile(tr, cache)
    assert (tw, th) in {(8, 8), (16, 16), (32, 32), (64, 64), (8, 16), (16, 8), (32, 4), (32, 8), (64, 4),
                        (8, 32), (16, 32), (32, 16)} and ms > 0
    assert cache.read_text().count("\n") == 1
    assert grt.rt_tune_tile(tr, cache) == (tw, th, pytest.approx(ms, rel=1e-5))
    assert cache.read_text().count("\n") == 1  # answered from the cache
    g = gpu_graph(tr, tile=(tw, th))
    g.analyze()
    assert_csr_equal(g, tr)
    g.close()
    tr1 = tg.random_rects(grid=(4000,), n=800, rects=(1, 3), side=(1, 60), seed=32, ndim=1)
    tw1, th1, _ = grt.rt_tune_tile(tr1, None)
    assert th1 == 1 and tw1 in (128, 256, 512, 1024)


def test_exec_tuner_configures_the_graph_and_results_hold(tmp_path):
    ensure_built()
    cache = tmp_path / "tune.txt"
    tr = tg.taskbench(256, 60, "random", seed=3)
    g = gpu_graph(tr, body=grt.RT_BODY_SPIN, spin_iters=9)
    g.analyze()
    c = g.tune(cache)
    assert c["policy"] in (grt.RT_EXEC_RING, grt.RT_EXEC_OWNED)
    if c["policy"] == grt.RT_EXEC_RING:
        assert c["warps"] in (2, 4, 8) and c["claim"] in (1, 2, 4, 8, 16, 32)
        assert c["keep"] in (2, 4, 8, 16, 32, 64)
    else:  # owned chunks: only the grid is tuned
        assert c["warps"] in (1, 2, 4)
    assert c["trials"] >= 10 and c["blocks"] > 0 and c["ms"] > 0
    g.out.zero_()
    g.execute()
    g.sync()
    want = np.array([oracle.spin(j, 9) for j in range(tr.n)], np.uint32).view(np.int32)
    assert np.array_equal(g.out.cpu().numpy(), want)
    c2 = g.tune(cache)
    assert c2["trials"] == 0 and (c2["blocks"], c2["warps"], c2["claim"], c2["keep"], c2["policy"]) == \
        (c["blocks"], c["warps"], c["claim"], c["keep"], c["policy"])
    g.close()


def test_batch_tuner_shape_runs_the_batch_correctly():
    ensure_built()
    traces = [tg.taskbench(32 << (k % 3), 20 + k, tg.PATTERNS[k % 3], seed=k) for k in range(12)]
    graphs = []
    for tr in traces:
        g = gpu_graph(tr, body=grt.RT_BODY_SPIN, spin_iters=13)
        g.analyze()
        graphs.append(g)
    batch = grt.Batch(graphs)
    c = batch.tune(replays=2)
    assert c["trials"] >= 10
    for g in graphs:
        g.out.zero_()
    batch.execute(replays=3, blocks=c["blocks"], warps=c["warps"], claim=c["claim"], keep=c["keep"])
    batch.sync()
    assert batch.counters()["tasks"] == 3 * sum(t.n for t in traces)
    for tr, g in zip(traces, graphs):
        want = np.array([oracle.spin(j, 13) for j in range(tr.n)], np.uint32).view(np.int32)
        assert np.array_equal(g.out.cpu().numpy(), want), tr.name
    batch.close()
    for g in graphs:
        g.close()
