"""Parity at the full sizes of the workloads, in the launch configurations
the benchmark uses: whole results against the oracle where it can take them
(the 1M-launch trace through the threaded interval-map oracle), element by
element on what it computes one by one elsewhere, and properties that hold
at any size on everything (edges point forward in program order, rows sorted
and unique, in-degrees equal column counts, every task of every replay ran)."""
import os

import numpy as np
import pytest

import oracle
from paper_2508_16522_gb300 import grt
from paper_2508_16522_gb300 import tracegen as tg

import oracle_pool
from gpu_helpers import ensure_built, gpu_graph

pytestmark = pytest.mark.gpu


def check_csr_invariants(n, rp, col, ind):
    rp = rp.astype(np.int64)
    assert rp[0] == 0 and rp[-1] == len(col) and np.all(np.diff(rp) >= 0)
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    col = col.astype(np.int64)
    assert np.all(col > src), "an edge does not point forward in program order"
    same = src[1:] == src[:-1]
    assert np.all(col[1:][same] > col[:-1][same]), "a row is not sorted and unique"
    assert np.array_equal(ind.astype(np.int64), np.bincount(col, minlength=n)), "indeg differs from column counts"
    return src, col


@pytest.fixture(scope="module")
def rects_4096():
    """The 1M-launch 4096^2 trace and its CSR from the interval-map oracle, which
    runs the per-cell rule row by row on every host core (pinned on the CPU to
    the per-cell oracle on downsized traces of this workload)."""
    tr = tg.random_rects(grid=(4096, 4096), n=1_000_000, seed=0)
    return tr, oracle.analyze_intervals(tr, os.cpu_count() or 1)


@pytest.mark.parametrize("tile", [(16, 16), (32, 32)])
def test_random_rects_4096_full_size_whole_csr(rects_4096, tile):
    """1M launches of 1-4 rects (sides log-uniform 16..1024) on 4096^2, at the
    library's default tile and at the one the benchmark uses: the WHOLE CSR
    (row_ptr, all 24,051,083 columns, in-degrees) equals the oracle's byte for
    byte."""
    ensure_built()
    tr, (rp_o, col_o) = rects_4096
    g = gpu_graph(tr, tile=tile, defer_check=True)
    g.analyze()
    rp, col, ind = g.csr()
    g.close()
    check_csr_invariants(tr.n, rp, col, ind)
    assert len(col) == len(col_o) == 24_051_083
    assert np.array_equal(rp.astype(np.int64), rp_o)
    assert np.array_equal(col, col_o)
    assert np.array_equal(ind.astype(np.int64), np.bincount(col_o, minlength=tr.n))


@pytest.fixture(scope="module")
def batch_digests():
    """The oracle's CSR and its CHECK state and outputs after 20 sequential runs,
    as digests, for every graph of the 4096-graph batch (spawned processes over
    the host's cores)."""
    return oracle_pool.batch_check_digests(4096, seed=0, runs=20)


def test_batched_full_size_every_graph(batch_digests):
    """4096 Task Bench graphs (sizes log-uniform 64..65536) in one persistent
    launch with 20 replays, as the benchmark runs them, every graph on the
    order-sensitive CHECK body: every graph's CSR equals the oracle's, and its
    state and outputs after the launch equal the oracle's after 20 sequential
    runs; the launch ran every task of every replay."""
    ensure_built()
    traces = tg.batch_graphs(4096, seed=0)
    graphs = []
    for tr in traces:
        g = gpu_graph(tr, body=grt.RT_BODY_CHECK)
        g.analyze()
        graphs.append(g)
    batch = grt.Batch(graphs)
    batch.execute(replays=20)
    batch.sync()
    c = batch.counters()
    total = sum(t.n for t in traces)
    assert c["tasks"] == 20 * total, c
    for k, (tr, g) in enumerate(zip(traces, graphs)):
        rp, col, ind = g.csr()
        check_csr_invariants(tr.n, rp, col, ind)
        want_csr, want_body = batch_digests[k]
        assert oracle_pool.csr_digest(rp, col) == want_csr, tr.name
        st = g.state.cpu().numpy()[:tr.n_cells]
        out = g.out.cpu().numpy()[:tr.n]
        assert oracle_pool.digest(st, out) == want_body, tr.name
    batch.close()
    for g in graphs:
        g.close()


def test_served_full_size_stream():
    """2000 requests of the served workload (Poisson at 50k graphs/s, sizes
    log-uniform 32..16384, dense rects on 1024^2) through the server as the
    benchmark configures it, results kept. All complete; every request's CSR
    equals the interval-map oracle's for that request alone, and its SPIN
    outputs are those of its own task ids."""
    ensure_built()
    reqs = tg.served_stream(2000, rate_per_s=50_000.0, seed=0)
    srv = grt.Server(2, [0, 0], [1023, 1023], body=grt.RT_BODY_SPIN, spin_iters=5, budget_bytes=8 << 30,
                     max_inflight=512, max_tasks=16384, workers=4, tile=(16, 16), max_batch=64, keep_results=True)
    tickets = [srv.submit(r.trace) for r in reqs]
    srv.drain(600_000_000_000)
    infos = [srv.poll(t) for t in tickets]
    assert all(i["state"] == 3 for i in infos)
    # a SPIN output depends only on the task's id within its request
    spin_all = np.array([oracle.spin(j, 5) for j in range(16384)], np.uint32).view(np.int32)
    threads = os.cpu_count() or 1
    for r, t, i in zip(reqs, tickets, infos):
        rp, col, out = srv.result(t, i["n_tasks"], i["n_edges"], with_out=True)
        assert np.array_equal(out, spin_all[:r.trace.n])
        rp_o, col_o = oracle.analyze_intervals(r.trace, threads)
        assert np.array_equal(rp.astype(np.int64), rp_o) and np.array_equal(col, col_o), r.trace.name
    srv.close()


def test_batched_full_size_stacked_capture(batch_digests):
    """The benchmark's capture of the batched workload: all 4096 graphs stacked
    in bands of one domain and analysed ONCE. Every graph's part of the CSR
    stays inside the graph and equals the graph's own oracle CSR; the stacked
    batch runs every task of 20 replays."""
    ensure_built()
    traces = tg.batch_graphs(4096, seed=0)
    st, off = tg.stack_bands(traces, name="batch")
    g = gpu_graph(st, tile=(8, 8), defer_check=True)
    g.analyze()
    rp, col, ind = g.csr()
    src, col64 = check_csr_invariants(st.n, rp, col, ind)
    graph_of = np.searchsorted(off, np.arange(st.n), side="right") - 1
    assert np.array_equal(graph_of[src], graph_of[col64]), "an edge joins two graphs"
    for k in range(len(traces)):
        a, b = int(off[k]), int(off[k + 1])
        got = oracle_pool.csr_digest(rp[a:b + 1].astype(np.int64) - int(rp[a]), col[rp[a]:rp[b]] - a)
        assert got == batch_digests[k][0], traces[k].name
    batch = grt.Batch.stacked(g, off)
    batch.execute(replays=20)
    batch.sync()
    assert batch.counters()["tasks"] == 20 * st.n
    batch.close()
    g.close()
