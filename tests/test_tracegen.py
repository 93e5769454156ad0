"""Seeded generators: determinism and the shapes/distributions of the workloads."""
import math

import numpy as np

from paper_2508_16522_gb300 import tracegen as tg


def _same(a, b):
    for f in ("req_off", "lo", "hi", "priv"):
        assert np.array_equal(getattr(a, f), getattr(b, f))


def test_determinism():
    _same(tg.random_rects(grid=(256, 256), n=5000, seed=7), tg.random_rects(grid=(256, 256), n=5000, seed=7))
    _same(tg.taskbench(64, 30, "random", seed=2), tg.taskbench(64, 30, "random", seed=2))
    a = tg.random_rects(grid=(256, 256), n=5000, seed=7)
    b = tg.random_rects(grid=(256, 256), n=5000, seed=8)
    assert not np.array_equal(a.lo, b.lo)


def test_random_rects_distribution():
    tr = tg.random_rects(grid=(4096, 4096), n=200_000, seed=0)
    counts = np.diff(tr.req_off)
    assert counts.min() == 1 and counts.max() == 4
    assert abs(counts.mean() - 2.5) < 0.02
    side = tr.hi - tr.lo + 1
    assert side.min() >= 16 and side.max() <= 1024
    # log-uniform: median of log side ~ midpoint of [ln 16, ln 1025]
    mid = 0.5 * (math.log(16) + math.log(1025))
    assert abs(np.median(np.log(side + 0.5)) - mid) < 0.05
    assert (tr.lo >= 0).all() and (tr.hi <= 4095).all()
    frac = np.bincount(tr.priv, minlength=3) / tr.n_rects
    assert np.allclose(frac, [0.6, 0.3, 0.1], atol=0.01)


def test_taskbench_shapes():
    for p, k in (("stencil", None), ("butterfly", 2), ("random", 5)):
        e = tg.taskbench(128, 20, p, encode="explicit")
        assert e.n == 128 * 20
        pc = np.diff(e.pred_off)
        assert (pc[:128] == 0).all()
        if k:
            assert (pc[128:] == k).all()
        t = np.repeat(np.arange(20), 128)
        for j in range(128, e.n):
            ps = e.pred[e.pred_off[j]:e.pred_off[j + 1]]
            assert (ps // 128 == t[j] - 1).all()  # only from step t-1
            assert len(set(ps.tolist())) == len(ps)  # distinct
    b = tg.taskbench(128, 20, "butterfly", encode="explicit")
    j = 5 * 128 + 9  # t = 5, i = 9: partner 9 ^ 2^(5 mod 7) = 9 ^ 32 = 41
    assert sorted(b.pred[b.pred_off[j]:b.pred_off[j + 1]].tolist()) == [4 * 128 + 9, 4 * 128 + 41]


def test_batch_graph_shapes():
    for n in (64, 100, 1000, 65536):
        w, s = tg.batch_graph_shape(n)
        assert 8 <= w <= 1024 and w * s <= n and s >= 1
    gs = tg.batch_graphs(16, seed=1)
    assert len(gs) == 16
    assert all(64 // 2 <= g.n <= 65536 for g in gs)


def test_served_stream_poisson():
    reqs = tg.served_stream(2000, rate_per_s=50_000.0, n_range=(32, 64), seed=3)
    gaps = np.diff([r.arrival_ns for r in reqs])
    assert abs(gaps.mean() / 1e9 - 1 / 50_000.0) < 0.1 / 50_000.0


def test_stack_bands_keeps_each_trace_to_itself():
    """The oracle on traces stacked in bands finds exactly each trace's own
    edges, moved by its task offset: no rectangle of one meets another's."""
    import oracle
    trs = [tg.random_rects(grid=(30 + 7 * k, 20 + 3 * k), n=120 + 40 * k, rects=(1, 3), side=(1, 12), seed=40 + k)
           for k in range(4)] + [tg.taskbench(16, 9, "butterfly", seed=1)]
    st, off = tg.stack_bands(trs)
    assert off[-1] == st.n and st.n == sum(t.n for t in trs)
    s, d = oracle.analyze(st)
    got = set(zip(s.tolist(), d.tolist()))
    want = set()
    for k, t in enumerate(trs):
        a, b = oracle.analyze(t)
        want |= set(zip((a + off[k]).tolist(), (b + off[k]).tolist()))
    assert got == want
