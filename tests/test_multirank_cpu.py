"""The multi-process path on CPU (gloo, world size 2): the job's time is the
slowest rank's; under torchrun only rank 0 prints the result line; and
independent graphs split across ranks by footprint (a batch largest first, a
served stream in arrival order) are each taken by exactly one rank, the shares
are balanced, and the union of what the ranks compute for their shares equals
what one rank computes for all of them."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    q.put((rank, bench.max_over_ranks(10.0 + 5.0 * rank, "cpu")))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    assert got == {0: 15.0, 1: 15.0}


def _batch_rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import oracle_pool
    from paper_2508_16522_gb300 import shard
    from paper_2508_16522_gb300 import tracegen as tg
    import oracle
    traces = tg.batch_graphs(96, n_range=(64, 4096), seed=3)
    share = shard.my_share([shard.footprint(t) for t in traces], world, rank)
    mine = {}
    for k in share:
        s, d = oracle.analyze(traces[k])
        rp, col = oracle.csr_from_pairs(traces[k].n, s, d)
        mine[k] = oracle_pool.csr_digest(rp, col)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    load = sum(shard.footprint(traces[k]) for k in share)
    loads = [None] * world
    dist.all_gather_object(loads, load)
    q.put((rank, gathered, loads))
    dist.barrier()
    dist.destroy_process_group()


def test_batch_split_across_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_batch_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    got = dict((r, (g, l)) for r, g, l in (q.get(timeout=10) for _ in range(2)))
    gathered, loads = got[0]
    assert got[1][0] == gathered and got[1][1] == loads  # every rank sees the same union
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import oracle
    import oracle_pool
    from paper_2508_16522_gb300 import shard
    from paper_2508_16522_gb300 import tracegen as tg
    traces = tg.batch_graphs(96, n_range=(64, 4096), seed=3)
    keys = [k for part in gathered for k in part]
    assert sorted(keys) == list(range(len(traces))), "a graph was taken by no rank or by two"
    union = {k: v for part in gathered for k, v in part.items()}
    for k, tr in enumerate(traces):  # one rank computing everything gives the same
        s, d = oracle.analyze(tr)
        assert union[k] == oracle_pool.csr_digest(*oracle.csr_from_pairs(tr.n, s, d))
    fps = [shard.footprint(t) for t in traces]
    assert sum(loads) == sum(fps)
    assert max(loads) - min(loads) <= max(fps)  # greedy largest-first balance


def _served_rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import oracle_pool
    from paper_2508_16522_gb300 import shard
    from paper_2508_16522_gb300 import tracegen as tg
    import oracle
    reqs = tg.served_stream(80, n_range=(32, 512), seed=5)
    share = shard.my_arrivals([shard.footprint(r.trace) for r in reqs], world, rank)
    mine = {}
    for k in share:
        tr = reqs[k].trace
        s, d = oracle.analyze(tr)
        mine[k] = oracle_pool.csr_digest(*oracle.csr_from_pairs(tr.n, s, d))
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    loads = [None] * world
    dist.all_gather_object(loads, sum(shard.footprint(reqs[k].trace) for k in share))
    q.put((rank, gathered, loads, share))
    dist.barrier()
    dist.destroy_process_group()


def test_served_stream_split_across_two_gloo_ranks():
    """Requests of a served stream placed in arrival order: each is taken by
    exactly one rank, every rank's share keeps the arrival order, the shares
    differ by at most the largest request, and the union of the ranks' CSRs
    equals one rank computing all of them."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_served_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    got = {r: (g, l, sh) for r, g, l, sh in (q.get(timeout=10) for _ in range(2))}
    gathered, loads, _ = got[0]
    assert got[1][0] == gathered and got[1][1] == loads
    for r in range(2):
        assert got[r][2] == sorted(got[r][2])  # arrival order kept
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import oracle
    import oracle_pool
    from paper_2508_16522_gb300 import shard
    from paper_2508_16522_gb300 import tracegen as tg
    reqs = tg.served_stream(80, n_range=(32, 512), seed=5)
    keys = [k for part in gathered for k in part]
    assert sorted(keys) == list(range(len(reqs))), "a request was taken by no rank or by two"
    union = {k: v for part in gathered for k, v in part.items()}
    for k, r in enumerate(reqs):
        s, d = oracle.analyze(r.trace)
        assert union[k] == oracle_pool.csr_digest(*oracle.csr_from_pairs(r.trace.n, s, d))
    fps = [shard.footprint(r.trace) for r in reqs]
    assert sum(loads) == sum(fps)
    assert max(loads) - min(loads) <= max(fps)


def _served_combine_rank(rank, world, port, fail_rank, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench

    def leg(grt, world, rank):  # one rank's share, as run_served reports it
        if rank == fail_rank:
            raise RuntimeError("server start failed")
        return {"span_s": 1.0 + rank, "requests": 10 * (rank + 1), "tasks": 1000 * (rank + 1),
                "latency_ms": {"p50": 5.0 + rank, "p99": 9.0 + rank}, "analysis_ms": {"p50": 2.0 * (rank + 1)}}

    q.put((rank, bench.run_served_split(None, world, rank, device="cpu", leg=leg)))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("fail_rank", [-1, 1])
def test_served_split_combines_ranks_and_survives_a_failed_rank(fail_rank):
    """The served leg over two ranks: all requests over the slowest rank's span
    (sums and maxima); when one rank's leg fails, both ranks still finish (no
    rank waits for the failed one) and both report the failure."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_served_combine_rank, args=(r, 2, port, fail_rank, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    if fail_rank < 0:
        for r in range(2):
            d = got[r]
            assert d["requests"] == 30 and d["tasks"] == 3000 and d["span_s"] == 2.0
            assert d["achieved_graphs_per_s"] == 15.0 and d["latency_ms"]["p99"] == 10.0 and d["ranks"] == 2
    else:
        assert all("error" in got[r] for r in range(2))
        assert "server start failed" in got[fail_rank]["error"]


def test_arrival_order_assignment_properties():
    sys.path.insert(0, ROOT)
    from paper_2508_16522_gb300 import shard
    import numpy as np
    rng = np.random.default_rng(2)
    for world in (1, 2, 3, 4, 8):
        fp = rng.integers(1, 10_000, size=300)
        owner = shard.assign_in_arrival_order(fp, world)
        loads = np.bincount(owner, weights=fp, minlength=world)
        assert owner.min() >= 0 and owner.max() < world
        # greedy in arrival order: a request goes where the share is smallest,
        # so no share passes the smallest by more than the largest request
        assert loads.max() - loads.min() <= fp.max()
        for k in range(len(fp)):  # each request went to a smallest share at its arrival
            before = np.bincount(owner[:k], weights=fp[:k], minlength=world)
            assert before[owner[k]] == before.min() and owner[k] == int(np.argmin(before))
        assert sorted(k for r in range(world) for k in shard.my_arrivals(fp, world, r)) == list(range(300))
    assert shard.assign_in_arrival_order([], 2).tolist() == []
    with pytest.raises(ValueError):
        shard.assign_in_arrival_order([1], 0)


def test_assignment_properties():
    sys.path.insert(0, ROOT)
    from paper_2508_16522_gb300 import shard
    import numpy as np
    rng = np.random.default_rng(1)
    for world in (1, 2, 3, 4, 8):
        fp = rng.integers(1, 10_000, size=200)
        owner = shard.assign_by_footprint(fp, world)
        loads = np.bincount(owner, weights=fp, minlength=world)
        assert owner.min() >= 0 and owner.max() < world
        assert loads.max() - loads.min() <= fp.max()
        assert sorted(k for r in range(world) for k in shard.my_share(fp, world, r)) == list(range(200))
        assert np.array_equal(owner, shard.assign_by_footprint(fp, world))  # deterministic
    assert shard.assign_by_footprint([], 3).tolist() == []


def test_reference_arm_under_torchrun_prints_once():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "3", "--graph-steps", "20"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
