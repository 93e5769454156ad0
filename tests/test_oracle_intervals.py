"""Pins of the interval-map analysis and of the threaded Algorithm 1 executor
(oracle/interval.c, oracle/alg1.c), on the CPU.

The interval analysis restates the per-cell run rule over segments of equal
run state and splits rows over threads; it must give exactly the per-cell
oracle's edges (itself pinned by the brute force, closed forms and the
Fig. 6(c) fixture) on every trace both can run, for every thread count, and
exactly the pairwise brute force on the tiny traces. Plausible mistakes are
planted in a temporary copy of interval.c and each must fail a pin.

The threaded executor must run every task once, order every edge (its
tickets), and give the sequential results of the SPIN and COUNTER bodies.
"""
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from oracle import oracle as orc_mod
from paper_2508_16522_gb300 import tracegen as tg

from test_oracle_pins import as_set, brute_force_edges, tiny_traces

SRC = os.path.join(os.path.dirname(orc_mod.__file__), "interval.c")


def b2_csr(tr):
    s, d = oracle.analyze(tr)
    return oracle.csr_from_pairs(tr.n, s, d)


def same_csr(a, b):
    return np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def csr_pairs(rp, col):
    src = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    return set(zip(src.tolist(), col.tolist()))


def medium_traces():
    out = []
    for seed in range(1, 7):
        out.append(tg.random_rects(grid=(64, 48), n=400, rects=(1, 4), side=(1, 20), seed=seed))
    for seed in range(7, 10):
        out.append(tg.random_rects(grid=(600,), n=300, rects=(1, 4), side=(1, 60), seed=seed, ndim=1))
    # many rectangles per task, long read runs, a task over the whole domain
    rng = np.random.default_rng(5)
    counts = [70] + [1] * 200 + [3] * 30
    R = sum(counts)
    lo = rng.integers(0, 30, size=(R, 2))
    hi = np.minimum(lo + rng.integers(0, 8, size=(R, 2)), 31)
    pv = np.where(np.arange(R) < 270, 0, rng.integers(0, 3, size=R)).astype(np.uint8)
    lo[70] = [0, 0]
    hi[70] = [31, 31]
    pv[70] = 1
    out.append(tg._finish(2, [0, 0], [31, 31], counts, lo.reshape(-1), hi.reshape(-1), pv, name="long_runs"))
    # an offset domain
    tr = tg.random_rects(grid=(40, 30), n=200, rects=(1, 3), side=(1, 12), seed=11)
    out.append(tg._finish(2, [-17, 1000], [22, 1029], np.diff(tr.req_off), (tr.lo + [-17, 1000]).reshape(-1),
                          (tr.hi + [-17, 1000]).reshape(-1), tr.priv, name="offset"))
    return out


@pytest.mark.parametrize("threads", [1, 3])
def test_equals_brute_force_on_tiny_traces(threads):
    for tr in tiny_traces():
        rp, col = oracle.analyze_intervals(tr, threads)
        assert csr_pairs(rp, col) == brute_force_edges(tr), tr.name


@pytest.mark.parametrize("threads", [1, 2, 5, 8])
def test_equals_per_cell_oracle(threads):
    for tr in medium_traces():
        assert same_csr(oracle.analyze_intervals(tr, threads), b2_csr(tr)), (tr.name, threads)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_equals_per_cell_oracle_on_downsized_random_rects(seed):
    """The 1M-launch 4096^2 workload scaled down (512^2, 10^4 launches, sides
    log-uniform 2..128): the per-cell oracle finishes in seconds here."""
    tr = tg.random_rects(grid=(512, 512), n=10_000, side=(2, 128), seed=seed)
    want = b2_csr(tr)
    for threads in (1, 8):
        assert same_csr(oracle.analyze_intervals(tr, threads), want), threads


def test_closed_forms_and_explicit_preds():
    # 1-D stencil: E = 2985 with the hand-derived edge set
    tr = tg.stencil_1d()
    rp, col = oracle.analyze_intervals(tr, 4)
    want = set()
    for t in range(100):
        for i in range(16):
            if i >= 1:
                want.add((16 * t + i - 1, 16 * t + i))
            if i <= 14 and t >= 1:
                want.add((16 * (t - 1) + i + 1, 16 * t + i))
    assert csr_pairs(rp, col) == want
    # Task Bench: region encoding equals the generated pred lists
    for pattern, e in (("stencil", 39 * (3 * 256 - 2)), ("butterfly", 39 * 512), ("random", 39 * 1280)):
        reg = tg.taskbench(256, 40, pattern, seed=2)
        exp = tg.taskbench(256, 40, pattern, seed=2, encode="explicit")
        a = oracle.analyze_intervals(reg, 3)
        b = oracle.analyze_intervals(exp, 3)
        assert len(a[1]) == e and same_csr(a, b), pattern
    # Fig. 6(c): explicit predecessors only
    rp, col = oracle.analyze_intervals(tg.fig6_fixture(), 2)
    assert csr_pairs(rp, col) == {(0, 1), (0, 2), (1, 3), (2, 3)}


def test_edge_cases():
    empty = tg._finish(2, [0, 0], [7, 7], np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0, np.int64),
                       np.zeros(0, np.uint8))
    rp, col = oracle.analyze_intervals(empty, 4)
    assert rp.tolist() == [0] and len(col) == 0
    rectless = tg._finish(2, [0, 0], [7, 7], np.zeros(5, np.int64), np.zeros(0, np.int64), np.zeros(0, np.int64),
                          np.zeros(0, np.uint8))
    rp, col = oracle.analyze_intervals(rectless, 4)
    assert rp.tolist() == [0] * 6 and len(col) == 0
    # one cell, more threads than rows and columns
    one = tg._finish(1, [3], [3], np.ones(5), np.full(5, 3, np.int64), np.full(5, 3, np.int64),
                     np.array([1, 0, 0, 2, 1], np.uint8))
    rp, col = oracle.analyze_intervals(one, 8)
    assert csr_pairs(rp, col) == brute_force_edges(one)


MUTANTS = {
    # a joining task takes edges from the current run instead of the one before
    "join_uses_current_run": ("if (emit_list(w, s->prev, j)) return -1;", "if (emit_list(w, s->cur, j)) return -1;"),
    # writes join a run of writes
    "writes_form_runs": ("if (s->cur && s->kind == p && p != K_WRITE) {", "if (s->cur && s->kind == p) {"),
    # neighbours merged when only their current runs agree
    "merge_ignores_previous_run": ("return a->kind == b->kind && a->cur == b->cur && a->prev == b->prev;",
                                   "return a->kind == b->kind && a->cur == b->cur;"),
    # read + reduce on one cell treated as read (O1)
    "combine_read_reduce": ("if (have == add && add != K_WRITE) return add;",
                            "if (have != K_WRITE && add != K_WRITE) return have;"),
    # one extended run reused for a segment whose run differs
    "memo_ignores_input": ("if (memo_in == s->cur && memo_out) {", "if (memo_out) {"),
    # the piece's right end not cut off from the rest of the segment
    "no_right_split": ("if (r + 1 <= row_end && row_split(row, r + 1) < 0) return -1;", "if (0) return -1;"),
    # a pair suppressed once its source was seen for any target
    "stamp_ignores_target": ("if (w->stamp[m->task] != j) {", "if (w->stamp[m->task] < 0) {"),
    # a row band ends one row early
    "band_short_by_one": ("w->ybnd[nb++] = (y1 > yb ? yb : y1) + 1;", "w->ybnd[nb++] = (y1 > yb ? yb : y1);"),
    # explicit predecessors dropped
    "drop_explicit_preds": ("if (ok && pred_off) {", "if (0) {"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "mut.c")
        so = os.path.join(d, "libmut.so")
        open(c, "w").write(src.replace(old, new))
        # the mutant library also needs the wrapper's other entry points
        base = [os.path.join(os.path.dirname(SRC), f) for f in ("oracle.c", "alg1.c")]
        subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", so, c] + base + ["-lm"])
        cases = tiny_traces() + [tg.stencil_1d(16, 6), tg.fig6_fixture()]
        wrong = 0
        for tr in cases:
            rp, col = oracle.analyze_intervals(tr, 2, lib_path=so)
            if csr_pairs(rp, col) != brute_force_edges(tr):
                wrong += 1
        for tr in medium_traces():
            if not same_csr(oracle.analyze_intervals(tr, 3, lib_path=so), b2_csr(tr)):
                wrong += 1
        assert wrong > 0, f"mutant {name} survived every pin"


# ---------------------------------------------------------------------------
# threaded Algorithm 1
# ---------------------------------------------------------------------------
def check_tickets(n, rp, col, tk):
    t = tk.reshape(-1, 2).astype(np.int64)
    assert sorted(t.reshape(-1).tolist()) == list(range(2 * n)), "a task did not run exactly once"
    assert np.all(t[:, 0] < t[:, 1])
    src = np.repeat(np.arange(n), np.diff(rp))
    assert np.all(t[src, 1] < t[col, 0]), "an edge was not respected"


@pytest.mark.parametrize("threads", [1, 2, 8])
def test_alg1_orders_every_edge(threads):
    for tr in medium_traces()[:6] + [tg.taskbench(64, 50, "random", seed=1), tg.fig6_fixture()]:
        rp, col = b2_csr(tr)
        for _ in range(3):
            _, _, tk, _ = oracle.alg1_run(tr.n, rp, col, threads, tickets=True)
            check_tickets(tr.n, rp, col, tk)


def test_alg1_bodies():
    tr = tg.stencil_1d()
    rp, col = b2_csr(tr)
    st, _, _, _ = oracle.alg1_run(tr.n, rp, col, 8, body=oracle.BODY_COUNTER, body_arg=tr.body_arg,
                                  state=np.zeros(16, np.int32))
    assert st.tolist() == [100] * 16
    tb = tg.taskbench(128, 30, "butterfly")
    rp, col = b2_csr(tb)
    _, out, _, ns = oracle.alg1_run(tb.n, rp, col, 4, body=oracle.BODY_SPIN, spin_iters=37)
    want = np.array([oracle.spin(v, 37) for v in range(tb.n)], np.uint32).view(np.int32)
    assert np.array_equal(out[:tb.n], want) and ns > 0


def test_alg1_full_size_taskbench():
    """A full 1024 x 1000 Task Bench graph (1.02M tasks) on every host core:
    every task runs once and every edge is ordered."""
    tr = tg.taskbench(1024, 1000, "random")
    rp, col = oracle.analyze_intervals(tr, os.cpu_count() or 1)
    _, _, tk, _ = oracle.alg1_run(tr.n, rp, col, os.cpu_count() or 1, tickets=True)
    check_tickets(tr.n, rp, col, tk)
