"""Parity at the full sizes of the workloads, in the launch configurations
the benchmark uses. The oracle cannot take these whole, so each test checks
what it can compute one by one (windows of the grid, sampled graphs, the
smallest requests) element by element, and properties that hold at any
size on everything (edges point forward in program order, rows sorted and
unique, in-degrees equal column counts, every task of every replay ran)."""
import numpy as np
import pytest

import oracle
from paper_2508_16522_gb300 import grt
from paper_2508_16522_gb300 import tracegen as tg

from gpu_helpers import ensure_built, gpu_graph, oracle_csr
from windows import clip_to_window

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


def test_random_rects_4096_full_size_windows():
    """1M launches of 1-4 rects (sides log-uniform 16..1024) on 4096^2, the
    library's default tiling. Three 64x64 windows: every edge the oracle finds
    in a window is in the GPU graph, and tasks wholly inside a window have
    exactly the oracle's in- and out-edges."""
    ensure_built()
    tr = tg.random_rects(grid=(4096, 4096), n=1_000_000, seed=0)
    g = gpu_graph(tr, defer_check=True)
    g.analyze()
    rp, col, ind = g.csr()
    g.close()
    n = tr.n
    src, col = check_csr_invariants(n, rp, col, ind)
    assert 10_000_000 <= len(col) <= 40_000_000
    keys = src * n + col  # ascending: rows in order, columns ascending
    by_dst = np.argsort(col, kind="stable")
    col_sorted = col[by_dst]
    rng = np.random.default_rng(0)
    inside_checked = 0
    for _ in range(3):
        wx, wy = (int(v) for v in rng.integers(0, 4096 - 64, 2))
        sub, ids, inside = clip_to_window(tr, [wx, wy], [wx + 63, wy + 63])
        s, d = oracle.analyze(sub)
        wkeys = ids[s].astype(np.int64) * n + ids[d]
        pos = np.searchsorted(keys, wkeys)
        assert np.all(pos < len(keys)) and np.array_equal(keys[np.minimum(pos, len(keys) - 1)], wkeys)
        for k in np.nonzero(inside)[0]:
            t = int(ids[k])
            mine = d == k
            want_in = np.sort(ids[s[mine]])
            a, b = np.searchsorted(col_sorted, [t, t + 1])
            assert np.array_equal(np.sort(src[by_dst[a:b]]), want_in), t
            want_out = np.sort(ids[d[s == k]])
            assert np.array_equal(col[rp[t]:rp[t + 1]], want_out), t
            inside_checked += 1
    assert inside_checked >= 3


def test_batched_full_size_sampled_graphs():
    """4096 Task Bench graphs (sizes log-uniform 64..65536) in one persistent
    launch with 20 replays, as the benchmark runs them. Every 128th graph runs
    the order-sensitive CHECK body and must end in the oracle's state after
    20 sequential runs; every graph's CSR is checked for the invariants, the
    sampled ones against the oracle, and the launch must have run every task
    of every replay."""
    ensure_built()
    traces = tg.batch_graphs(4096, seed=0)
    sampled = set(range(0, 4096, 128)) | {int(np.argmax([t.n for t in traces]))}
    graphs = []
    for k, tr in enumerate(traces):
        body = grt.RT_BODY_CHECK if k in sampled else grt.RT_BODY_EMPTY
        g = gpu_graph(tr, body=body)
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
        if k in sampled:
            rp_o, col_o, _ = oracle_csr(tr)
            assert np.array_equal(rp.astype(np.int64), rp_o) and np.array_equal(col, col_o), tr.name
            st = out = None
            for _ in range(20):
                st, out = oracle.run_bodies(tr, oracle.oracle.BODY_CHECK, state=st)
            assert np.array_equal(g.state.cpu().numpy(), st), tr.name
            assert np.array_equal(g.out.cpu().numpy(), out), tr.name
    batch.close()
    for g in graphs:
        g.close()


def test_served_full_size_stream():
    """2000 requests of the served workload (Poisson at 50k graphs/s, sizes
    log-uniform 32..16384, dense rects on 1024^2) through the server as the
    benchmark configures it, results kept. All complete; every result passes
    the invariants; the smallest requests match the oracle exactly."""
    ensure_built()
    reqs = tg.served_stream(2000, rate_per_s=50_000.0, seed=0)
    srv = grt.Server(2, [0, 0], [1023, 1023], body=grt.RT_BODY_SPIN, spin_iters=5, budget_bytes=8 << 30,
                     max_inflight=512, max_tasks=16384, workers=4, tile=(16, 16), max_batch=64, keep_results=True)
    tickets = [srv.submit(r.trace) for r in reqs]
    srv.drain(600_000_000_000)
    infos = [srv.poll(t) for t in tickets]
    assert all(i["state"] == 3 for i in infos)
    order = np.argsort([r.trace.n for r in reqs])
    exact = set(order[:6].tolist())
    # a SPIN output depends only on the task's id within its request
    spin_all = np.array([oracle.spin(j, 5) for j in range(16384)], np.uint32).view(np.int32)
    for k, (r, t, i) in enumerate(zip(reqs, tickets, infos)):
        rp, col, out = srv.result(t, i["n_tasks"], i["n_edges"], with_out=True)
        check_csr_invariants(r.trace.n, rp, col, np.bincount(col, minlength=r.trace.n))
        assert np.array_equal(out, spin_all[:r.trace.n])
        if k in exact:
            rp_o, col_o, _ = oracle_csr(r.trace)
            assert np.array_equal(rp.astype(np.int64), rp_o) and np.array_equal(col, col_o)
    srv.close()


def test_batched_full_size_stacked_capture():
    """The benchmark's capture of the batched workload: all 4096 graphs stacked
    in bands of one domain and analysed ONCE. Every graph's part of the CSR
    passes the invariants and stays inside the graph; sampled graphs (every
    256th and the largest) equal their own oracle CSR; the stacked batch runs
    every task of 20 replays."""
    ensure_built()
    traces = tg.batch_graphs(4096, seed=0)
    st, off = tg.stack_bands(traces, name="batch")
    g = gpu_graph(st, tile=(8, 8), defer_check=True)
    g.analyze()
    rp, col, ind = g.csr()
    src, col64 = check_csr_invariants(st.n, rp, col, ind)
    graph_of = np.searchsorted(off, np.arange(st.n), side="right") - 1
    assert np.array_equal(graph_of[src], graph_of[col64]), "an edge joins two graphs"
    sampled = set(range(0, 4096, 256)) | {int(np.argmax([t.n for t in traces]))}
    for k in sorted(sampled):
        a, b = int(off[k]), int(off[k + 1])
        rp_o, col_o, _ = oracle_csr(traces[k])
        assert np.array_equal(rp[a:b + 1].astype(np.int64) - int(rp[a]), rp_o), traces[k].name
        assert np.array_equal(col[rp[a]:rp[b]] - a, col_o), traces[k].name
    batch = grt.Batch.stacked(g, off)
    batch.execute(replays=20)
    batch.sync()
    assert batch.counters()["tasks"] == 20 * st.n
    batch.close()
    g.close()
