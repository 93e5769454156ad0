"""Serving: requests analysed by worker threads and executed by one persistent
kernel that admits new graphs while others run. Each request's result in the
mix must equal its result alone: the canonical CSR, the SPIN outputs, and with
the order-sensitive CHECK body the request's final state and per-task outputs,
which equal the oracle's sequential run of that request only if every edge was
respected while it ran beside the others."""
import os
import time

import numpy as np
import pytest

import oracle
from paper_2508_16522_gb300 import grt
from paper_2508_16522_gb300 import tracegen as tg

from gpu_helpers import ensure_built, oracle_csr

pytestmark = pytest.mark.gpu

GRID = (128, 128)


def requests(k, seed, n_range=(32, 1500)):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(k):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        out.append(tg.random_rects(grid=GRID, n=n, rects=(1, 4), side=(2, 32), seed=seed * 1000 + i))
    return out


def check_all(srv, tickets, traces, spin_iters):
    for t, tr in zip(tickets, traces):
        info = srv.poll(t)
        assert info["state"] == 3, (tr.name, info)
        assert info["arrival_ns"] <= info["admit_ns"] <= info["posted_ns"] <= info["done_ns"]
        rp, col, out = srv.result(t, info["n_tasks"], info["n_edges"], with_out=True)
        rp_o, col_o, _ = oracle_csr(tr)
        assert np.array_equal(rp.astype(np.int64), rp_o) and np.array_equal(col, col_o), tr.name
        want = np.array([oracle.spin(j, spin_iters) for j in range(tr.n)], np.uint32).view(np.int32)
        assert np.array_equal(out, want), tr.name


def check_all_check_body(srv, tickets, traces):
    for t, tr in zip(tickets, traces):
        info = srv.poll(t)
        assert info["state"] == 3, (tr.name, info)
        rp, col, out = srv.result(t, info["n_tasks"], info["n_edges"], with_out=True)
        rp_o, col_o, _ = oracle_csr(tr)
        assert np.array_equal(rp.astype(np.int64), rp_o) and np.array_equal(col, col_o), tr.name
        st_o, out_o = oracle.run_bodies(tr, oracle.BODY_CHECK)
        assert np.array_equal(srv.result_state(t, tr.n_cells), st_o[:tr.n_cells]), tr.name
        assert np.array_equal(out, out_o[:tr.n]), tr.name


def test_check_body_burst_in_the_mix_equals_alone():
    """60 requests arriving at once, up to 16 running together beside later
    batches: each request's CHECK state and outputs equal its sequential run."""
    ensure_built()
    traces = requests(60, seed=21)
    srv = grt.Server(2, [0, 0], [GRID[0] - 1, GRID[1] - 1], body=grt.RT_BODY_CHECK, max_inflight=16,
                     max_tasks=2048, workers=4, keep_results=True, budget_bytes=2 << 30)
    tickets = [srv.submit(tr) for tr in traces]
    srv.drain(120_000_000_000)
    check_all_check_body(srv, tickets, traces)
    st = srv.stats()
    assert st["batched_requests"] == 60 and st["batches"] < 60, st
    srv.close()


def test_check_body_paced_offset_domain():
    """Paced arrivals that overlap in the kernel, on a domain that does not
    start at 0 (each request's band origin and cell indices are its own)."""
    ensure_built()
    lo, hi = np.array([5, -7]), np.array([5 + 95, -7 + 79])
    traces = []
    for i in range(24):
        tr = tg.random_rects(grid=(96, 80), n=100 + 37 * i, rects=(1, 4), side=(2, 24), seed=300 + i)
        traces.append(tg._finish(2, lo, hi, np.diff(tr.req_off), (tr.lo + lo).reshape(-1), (tr.hi + lo).reshape(-1),
                                 tr.priv, name=f"offset{i}"))
    srv = grt.Server(2, lo, hi, body=grt.RT_BODY_CHECK, max_inflight=8, max_tasks=1024, workers=3,
                     keep_results=True, max_batch=4)
    tickets = []
    for tr in traces:
        tickets.append(srv.submit(tr))
        time.sleep(0.0005)
    srv.drain(120_000_000_000)
    check_all_check_body(srv, tickets, traces)
    srv.close()


def test_check_body_one_dimensional():
    ensure_built()
    traces = [tg.random_rects(grid=(997,), n=int(n), rects=(1, 4), side=(1, 90), seed=170 + i, ndim=1)
              for i, n in enumerate((400, 37, 250, 1, 600, 128, 512, 77))]
    srv = grt.Server(1, [0], [996], body=grt.RT_BODY_CHECK, max_inflight=6, max_tasks=600, workers=2,
                     keep_results=True, max_batch=3)
    tickets = [srv.submit(tr) for tr in traces]
    srv.drain(120_000_000_000)
    check_all_check_body(srv, tickets, traces)
    srv.close()


def test_burst_in_the_mix_equals_alone():
    ensure_built()
    traces = requests(60, seed=1)
    srv = grt.Server(2, [0, 0], [GRID[0] - 1, GRID[1] - 1], body=grt.RT_BODY_SPIN, spin_iters=11,
                     max_inflight=16, max_tasks=2048, workers=4, keep_results=True, budget_bytes=2 << 30)
    tickets = [srv.submit(tr) for tr in traces]
    srv.drain(60_000_000_000)
    check_all(srv, tickets, traces, 11)
    st = srv.stats()
    # requests that waited together were analysed together
    assert st["batched_requests"] == 60 and st["batches"] < 60, st
    # the kernel keeps running: a second wave is admitted and executed too
    more = requests(20, seed=2)
    t2 = [srv.submit(tr) for tr in more]
    srv.drain(60_000_000_000)
    check_all(srv, t2, more, 11)
    srv.close()


def test_paced_arrivals_overlap_and_match():
    ensure_built()
    traces = requests(40, seed=3, n_range=(200, 2000))
    srv = grt.Server(2, [0, 0], [GRID[0] - 1, GRID[1] - 1], body=grt.RT_BODY_SPIN, spin_iters=200,
                     max_inflight=8, max_tasks=2048, workers=3, keep_results=True)
    tickets = []
    for tr in traces:
        tickets.append(srv.submit(tr))
        time.sleep(0.0005)
    srv.drain(60_000_000_000)
    check_all(srv, tickets, traces, 200)
    infos = [srv.poll(t) for t in tickets]
    # continuous batching: some request was admitted before an earlier one finished
    overlap = any(infos[i + 1]["admit_ns"] < infos[i]["done_ns"] for i in range(len(infos) - 1))
    assert overlap
    srv.close()


def test_small_budget_and_few_slots_serialise_but_stay_correct():
    ensure_built()
    traces = requests(12, seed=4, n_range=(100, 800))
    # each request's estimate is ~8 MB + ...: a 40 MB budget admits at most a few
    srv = grt.Server(2, [0, 0], [GRID[0] - 1, GRID[1] - 1], body=grt.RT_BODY_SPIN, spin_iters=5,
                     max_inflight=2, max_tasks=1024, workers=2, keep_results=True, budget_bytes=40 << 20)
    tickets = [srv.submit(tr) for tr in traces]
    srv.drain(60_000_000_000)
    check_all(srv, tickets, traces, 5)
    st = srv.stats()
    assert st["ledger_peak_bytes"] <= 40 << 20 and st["held_peak_bytes"] <= 40 << 20, st
    # a request larger than max_tasks is refused outright
    with pytest.raises(grt.GrtError) as e:
        srv.submit(tg.random_rects(grid=GRID, n=1500, rects=(1, 1), side=(2, 3), seed=10))
    assert e.value.status == grt.RT_ERR_INVALID
    srv.close()


def test_budget_bounds_the_bytes_held_under_a_burst():
    """A burst under a 128 MB budget, with one request whose analysis needs far
    more than its estimate (400 readers then 400 reducers of the whole domain:
    160k edges, each found in every tile). Its batch outgrows its cap, is
    admitted again with larger estimates and, once even the whole budget is
    not enough, fails with RT_ERR_BUDGET; the other requests give their results
    alone. The bytes the batch graphs may hold (caps and retained buffers) and
    the bytes they held after each analysis never pass the budget."""
    ensure_built()
    budget = 128 << 20
    K = 400
    full = np.array([[0, 0]] * (2 * K), np.int64)
    quad = tg._finish(2, [0, 0], [GRID[0] - 1, GRID[1] - 1], np.ones(2 * K), full.reshape(-1),
                      np.tile([GRID[0] - 1, GRID[1] - 1], 2 * K), np.array([0] * K + [2] * K, np.uint8), name="quad")
    ok = requests(24, seed=32, n_range=(100, 700))
    srv = grt.Server(2, [0, 0], [GRID[0] - 1, GRID[1] - 1], body=grt.RT_BODY_SPIN, spin_iters=3, max_inflight=8,
                     max_tasks=2048, workers=3, keep_results=True, budget_bytes=budget, max_batch=4)
    t_ok = [srv.submit(tr) for tr in ok[:12]]
    t_q = srv.submit(quad)
    t_ok += [srv.submit(tr) for tr in ok[12:]]
    srv.drain(120_000_000_000)
    check_all(srv, t_ok, ok, 3)
    info = srv.poll(t_q)
    assert info["state"] == 4 and info["status"] == grt.RT_ERR_BUDGET, info
    st = srv.stats()
    assert st["budget_retries"] >= 1, st
    assert 0 < st["ledger_peak_bytes"] <= budget, st
    assert 0 < st["held_peak_bytes"] <= budget, st
    srv.close()


def test_empty_request_and_budget_refusal():
    ensure_built()
    srv = grt.Server(2, [0, 0], [GRID[0] - 1, GRID[1] - 1], body=grt.RT_BODY_EMPTY, max_inflight=4,
                     max_tasks=4096, workers=1, keep_results=True, budget_bytes=16 << 20)
    empty = tg._finish(2, [0, 0], [GRID[0] - 1, GRID[1] - 1], np.zeros(0, np.int64), np.zeros(0, np.int64),
                       np.zeros(0, np.int64), np.zeros(0, np.uint8))
    t = srv.submit(empty)
    srv.drain(10_000_000_000)
    assert srv.poll(t)["state"] == 3
    big = tg.random_rects(grid=GRID, n=4000, rects=(4, 4), side=(2, 4), seed=11)
    with pytest.raises(grt.GrtError) as e:
        srv.submit(big)  # estimate (> 16 MB) can never fit the budget
    assert e.value.status == grt.RT_ERR_BUDGET
    srv.close()


def test_one_request_per_batch_gives_the_same_results():
    ensure_built()
    traces = requests(16, seed=5, n_range=(50, 400))
    srv = grt.Server(2, [0, 0], [GRID[0] - 1, GRID[1] - 1], body=grt.RT_BODY_SPIN, spin_iters=3,
                     max_inflight=8, max_tasks=512, workers=2, keep_results=True, max_batch=1)
    tickets = [srv.submit(tr) for tr in traces]
    srv.drain(60_000_000_000)
    check_all(srv, tickets, traces, 3)
    st = srv.stats()
    assert st["batches"] == 16 and st["batched_requests"] == 16, st
    srv.close()


def test_one_dimensional_requests_stack_along_x():
    ensure_built()
    traces = [tg.random_rects(grid=(997,), n=int(n), rects=(1, 4), side=(1, 90), seed=70 + i, ndim=1)
              for i, n in enumerate((400, 37, 250, 1, 600, 128))]
    srv = grt.Server(1, [0], [996], body=grt.RT_BODY_SPIN, spin_iters=7, max_inflight=6, max_tasks=600,
                     workers=1, keep_results=True, max_batch=4)
    tickets = [srv.submit(tr) for tr in traces]
    srv.drain(60_000_000_000)
    check_all(srv, tickets, traces, 7)
    srv.close()


def test_submit_rejects_rectangles_outside_the_domain():
    ensure_built()
    srv = grt.Server(2, [0, 0], [GRID[0] - 1, GRID[1] - 1], max_inflight=2, max_tasks=64, workers=1)
    bad = tg._finish(2, [0, 0], [GRID[0] - 1, GRID[1] + 9], np.array([1]), np.array([0, GRID[1]]),
                     np.array([3, GRID[1] + 2]), np.array([1], np.uint8))
    with pytest.raises(grt.GrtError) as e:
        srv.submit(bad)  # a rectangle past the domain would reach the next request's band
    assert e.value.status == grt.RT_ERR_INVALID
    srv.close()


_FRESH = r'''
import sys
sys.path.insert(0, sys.argv[1])
from paper_2508_16522_gb300 import grt, tracegen as tg
grt.load()
# nothing has run in this process: the server is the first user of the library,
# so every kernel its workers launch must have been loaded before its kernel
reqs = tg.served_stream(40, rate_per_s=50000.0, seed=3)
srv = grt.Server(2, [0, 0], [1023, 1023], body=grt.RT_BODY_EMPTY, budget_bytes=2 << 30, max_inflight=64,
                 max_tasks=16384, workers=2, tile=(16, 16), max_batch=16)
tickets = [srv.submit(r.trace) for r in reqs]
srv.drain(timeout_ns=60_000_000_000)
edges = [srv.poll(t)["n_edges"] for t in tickets]
srv.close()
print(sum(edges))
'''


def test_server_as_the_first_thing_a_process_runs():
    """A server created before any other call of the library analyses dense
    batches (all of the analysis kernels, the bucket CSR and the pair-key
    filter among them) while its kernel is resident. Run in a fresh process,
    bounded, and compared with the oracle's edge counts."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    ensure_built()
    out = subprocess.run([sys.executable, "-c", _FRESH, root], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    want = sum(len(oracle_csr(r.trace)[1]) for r in tg.served_stream(40, rate_per_s=50000.0, seed=3))
    assert int(out.stdout.strip().splitlines()[-1]) == want
