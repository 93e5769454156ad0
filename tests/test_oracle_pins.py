"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* the paper's Fig. 6(c) four-task DAG (tests/golden/fig6c_simple_dag.txt)
* closed forms of the 1-D stencil and Task Bench graphs (derived by hand
  from the per-cell run rule, independent of the oracle's state machine)
* brute force on tiny traces: a *pairwise* restatement of the edge rule
  (edge i->j at cell c iff exactly one run boundary separates i and j in c's
  access sequence), computed with set-based privilege combination
* interference soundness (every edge joins two conflicting accesses) and
  completeness (every conflicting pair is connected by a path)
* executor: any topological order of the edges reproduces program-order
  bodies; dropping a needed edge is caught (mistake planted on the CPU)
* the SPIN body against the closed form of an affine recurrence
"""
import os

import numpy as np
import pytest

import oracle
from paper_2508_16522_gb300 import tracegen as tg

R, W, RED = 0, 1, 2
GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# independent restatements used only here
# ---------------------------------------------------------------------------
def cell_sequences(tr):
    """{cell: [(task, combined privilege), ...]} in program order, combining a
    task's rects by *sets*: {read} -> read, {reduce} -> reduce, else write."""
    ext = tr.extent()
    seqs = {}
    for j in range(tr.n):
        privs = {}
        for r in range(tr.req_off[j], tr.req_off[j + 1]):
            lo, hi = tr.lo[r], tr.hi[r]
            xs = range(int(lo[0] - tr.dom_lo[0]), int(hi[0] - tr.dom_lo[0]) + 1)
            ys = range(int(lo[1] - tr.dom_lo[1]), int(hi[1] - tr.dom_lo[1]) + 1) if tr.ndim == 2 else [0]
            for y in ys:
                for x in xs:
                    privs.setdefault(y * ext[0] + x, set()).add(int(tr.priv[r]))
        for c, s in privs.items():
            p = R if s == {R} else (RED if s == {RED} else W)
            seqs.setdefault(c, []).append((j, p))
    return seqs


def brute_force_edges(tr):
    """Pairwise form of the run rule: (i, j) is an edge iff at some cell exactly
    one run boundary lies between i and j (a boundary sits between two
    consecutive accesses unless both are reads or both are reduces)."""
    edges = set()
    for seq in cell_sequences(tr).values():
        kinds = [p for _, p in seq]
        bnd = [0] + [0 if (kinds[x] == kinds[x + 1] and kinds[x] != W) else 1 for x in range(len(seq) - 1)]
        pref = np.cumsum(bnd)
        for a in range(len(seq)):
            for b in range(a + 1, len(seq)):
                if pref[b] - pref[a] == 1:
                    edges.add((seq[a][0], seq[b][0]))
    if tr.pred_off is not None:
        for j in range(tr.n):
            for k in range(tr.pred_off[j], tr.pred_off[j + 1]):
                edges.add((int(tr.pred[k]), j))
    return edges


def interfering_pairs(tr):
    out = set()
    for seq in cell_sequences(tr).values():
        for a in range(len(seq)):
            for b in range(a + 1, len(seq)):
                pa, pb = seq[a][1], seq[b][1]
                if not (pa == pb and pa != W):
                    out.add((seq[a][0], seq[b][0]))
    return out


def closure_reach(n, edges):
    succ = [[] for _ in range(n)]
    for s, d in edges:
        succ[s].append(d)
    reach = [set() for _ in range(n)]
    for v in range(n - 1, -1, -1):
        for d in succ[v]:
            reach[v].add(d)
            reach[v] |= reach[d]
    return reach


def tiny_traces():
    out = []
    for seed in range(1, 41):
        ndim = 1 if seed % 4 == 0 else 2
        grid = (12,) if ndim == 1 else (7, 6)
        out.append(tg.random_rects(grid=grid, n=18 + seed % 7, rects=(1, 3), side=(1, 5),
                                   probs=(0.45, 0.35, 0.2), seed=seed, ndim=ndim))
    # exhaustive privilege mixes of three tasks on a single cell
    for a in range(3):
        for b in range(3):
            for c in range(3):
                for d in range(3):
                    lo = np.zeros((4, 1), np.int64)
                    out.append(tg._finish(1, [0], [0], np.ones(4), lo.reshape(-1), lo.reshape(-1),
                                          np.array([a, b, c, d], np.uint8), name=f"mix{a}{b}{c}{d}"))
    return out


def as_set(src, dst):
    return set(zip(src.tolist(), dst.tolist()))


# ---------------------------------------------------------------------------
# tests
# ---------------------------------------------------------------------------
def read_golden():
    edges, info = [], {}
    with open(os.path.join(GOLD, "fig6c_simple_dag.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, *v = line.split()
            if k == "edge":
                edges.append((int(v[0]), int(v[1])))
            else:
                info[k] = [int(x) for x in v]
    return edges, info


def test_fig6c_fixture_edges_roots_order():
    edges, info = read_golden()
    tr = tg.fig6_fixture()
    src, dst = oracle.analyze(tr)
    assert sorted(zip(src.tolist(), dst.tolist())) == edges
    rp, col = oracle.csr_from_pairs(tr.n, src, dst)
    indeg = np.bincount(dst, minlength=tr.n)
    assert indeg.tolist() == info["indeg"]
    assert np.flatnonzero(indeg == 0).tolist() == info["roots"]
    assert oracle.topo_order(tr.n, rp, col).tolist() == info["kahn_min_order"]


def test_stencil_1d_closed_form():
    """16 pieces x 100 steps, id = 16 t + i: edges are (i-1,t)->(i,t) for i>=1
    and (i+1,t-1)->(i,t) for i<=14, t>=1; 1500 + 1485 = 2985 edges."""
    P, T = 16, 100
    tr = tg.stencil_1d(P, T)
    got = as_set(*oracle.analyze(tr))
    want = set()
    for t in range(T):
        for i in range(P):
            if i >= 1:
                want.add((16 * t + i - 1, 16 * t + i))
            if i <= P - 2 and t >= 1:
                want.add((16 * (t - 1) + i + 1, 16 * t + i))
    assert len(want) == 2985
    assert got == want


def test_stencil_1d_counter_final_state():
    tr = tg.stencil_1d()
    state, _ = oracle.run_bodies(tr, oracle.oracle.BODY_COUNTER, state=np.zeros(16, np.int32))
    assert state.tolist() == [100] * 16


@pytest.mark.parametrize("pattern,k", [("stencil", None), ("butterfly", 2), ("random", 5)])
def test_taskbench_closed_forms(pattern, k):
    width, steps = 1024, 40
    reg = tg.taskbench(width, steps, pattern, seed=3)
    exp = tg.taskbench(width, steps, pattern, seed=3, encode="explicit")
    s1, d1 = oracle.analyze(reg)
    s2, d2 = oracle.analyze(exp)
    if pattern == "stencil":
        assert len(s1) == (steps - 1) * (3 * width - 2)
    else:
        assert len(s1) == (steps - 1) * width * k
    # region encoding and explicit preds give the identical CSR
    assert np.array_equal(s1, s2) and np.array_equal(d1, d2)
    # and those edges are exactly the generated pred lists
    want = set()
    for j in range(exp.n):
        for q in range(exp.pred_off[j], exp.pred_off[j + 1]):
            want.add((int(exp.pred[q]), j))
    assert as_set(s1, d1) == want
    # in-degree histogram is the pattern's
    indeg = np.bincount(d1, minlength=reg.n)
    assert (indeg[:width] == 0).all()
    if pattern != "stencil":
        assert (indeg[width:] == k).all()
    else:
        assert sorted(set(indeg[width:].tolist())) == [2, 3]


def test_taskbench_full_size_counts():
    """width 1024 x 1000 steps: E = 999*(3*1024-2), 999*2048, 999*5120."""
    want = {"stencil": 3_066_930, "butterfly": 2_045_952, "random": 5_114_880}
    for p, e in want.items():
        s, d = oracle.analyze(tg.taskbench(1024, 1000, p))
        assert len(s) == e
        assert (s < d).all()


def test_brute_force_pairwise_rule():
    for tr in tiny_traces():
        got = as_set(*oracle.analyze(tr))
        assert got == brute_force_edges(tr), tr.name


def test_soundness_and_completeness():
    for tr in tiny_traces():
        src, dst = oracle.analyze(tr)
        edges = as_set(src, dst)
        inter = interfering_pairs(tr)
        assert edges <= inter, tr.name  # sound
        reach = closure_reach(tr.n, edges)
        for i, j in inter:  # complete: every conflict ordered by a path
            assert j in reach[i], (tr.name, i, j)
        assert all(s < d for s, d in edges)  # forward in program order => acyclic


def test_explicit_preds_deduplicated():
    tr = tg._finish(2, [0, 0], [0, 0], np.zeros(3), np.zeros(0, np.int64), np.zeros(0, np.int64),
                    np.zeros(0, np.uint8), pred_counts=[0, 2, 3], pred=[0, 0, 1, 0, 1])
    s, d = oracle.analyze(tr)
    assert as_set(s, d) == {(0, 1), (0, 2), (1, 2)} and len(s) == 3


def largest_first_topo(n, rp, col):
    import heapq
    cnt = np.zeros(n, np.int64)
    np.add.at(cnt, col, 1)
    h = [-v for v in range(n) if cnt[v] == 0]
    heapq.heapify(h)
    out = []
    while h:
        v = -heapq.heappop(h)
        out.append(v)
        for e in range(rp[v], rp[v + 1]):
            cnt[col[e]] -= 1
            if cnt[col[e]] == 0:
                heapq.heappush(h, -int(col[e]))
    return np.array(out, np.int32)


def test_check_body_any_topological_order_matches_program_order():
    for seed in range(1, 25):
        tr = tg.random_rects(grid=(16, 12), n=60, rects=(1, 4), side=(1, 8), seed=seed)
        src, dst = oracle.analyze(tr)
        rp, col = oracle.csr_from_pairs(tr.n, src, dst)
        seq_state, seq_out = oracle.run_bodies(tr, oracle.oracle.BODY_CHECK)
        for order in (oracle.topo_order(tr.n, rp, col), largest_first_topo(tr.n, rp, col)):
            assert len(order) == tr.n
            st, out = oracle.run_bodies(tr, oracle.oracle.BODY_CHECK, order=order)
            assert np.array_equal(st, seq_state) and np.array_equal(out, seq_out)


def test_check_body_detects_a_dropped_edge():
    """Plant a mistake on the CPU: drop one edge, execute a topological order of
    the reduced graph that runs the edge's target first; CHECK must differ."""
    caught = 0
    for seed in range(1, 30):
        tr = tg.random_rects(grid=(10, 10), n=30, rects=(1, 2), side=(2, 6), seed=seed)
        src, dst = oracle.analyze(tr)
        seq_state, seq_out = oracle.run_bodies(tr, oracle.oracle.BODY_CHECK)
        # pick a RAW edge whose target can be hoisted: drop all edges into dst
        # from src and run dst right before src
        for e in range(len(src)):
            a, b = int(src[e]), int(dst[e])
            order = [v for v in range(tr.n) if v != b]
            order.insert(order.index(a), b)
            st, out = oracle.run_bodies(tr, oracle.oracle.BODY_CHECK, order=np.array(order, np.int32))
            if not (np.array_equal(st, seq_state) and np.array_equal(out, seq_out)):
                caught += 1
        assert caught > 0
    assert caught > 100


def affine_pow(a, c, n):
    """(a, c)^n under composition x -> a x + c (mod 2^32), by squaring."""
    M = 1 << 32
    ra, rc = 1, 0
    ba, bc = a, c
    while n:
        if n & 1:
            ra, rc = (ba * ra) % M, (ba * rc + bc) % M
        ba, bc = (ba * ba) % M, (ba * bc + bc) % M
        n >>= 1
    return ra, rc


def test_spin_body_closed_form():
    for x0 in (0, 1, 12345, 2**31 - 1, 2**32 - 7):
        for it in (0, 1, 2, 255, 256, 1000):
            A, C = affine_pow(1664525, 1013904223, it)
            assert oracle.spin(x0, it) == (A * x0 + C) % (1 << 32)


def round_to_binary32(q):
    """Bits of the binary32 value nearest to the rational q (ties to even);
    q is positive and in the normal range."""
    from fractions import Fraction
    assert q > 0
    e = q.numerator.bit_length() - q.denominator.bit_length()
    while Fraction(2) ** e > q:
        e -= 1
    while Fraction(2) ** (e + 1) <= q:
        e += 1
    m = q / Fraction(2) ** (e - 23)  # in [2^23, 2^24)
    fl = m.numerator // m.denominator
    rem = m - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    if fl == 1 << 24:
        fl, e = 1 << 23, e + 1
    return ((e + 127) << 23) | (fl - (1 << 23))


def test_fma_body_is_binary32_fused_multiply_add():
    """The FMA body against IEEE binary32 arithmetic written out with exact
    rationals: each step takes x * a + b exactly and rounds it once to the
    nearest float (ties to even); a = 0.999 and b = 0.25 as binary32."""
    from fractions import Fraction
    a = Fraction(float(np.float32(0.999)))
    b = Fraction(1, 4)
    for task in (0, 1, 7, 12345, 999_999, (1 << 24) + 1):
        x = Fraction(float(np.float32(task)))  # the task id rounded to binary32
        for it in range(0, 41):
            if it in (0, 1, 2, 3, 17, 40):
                want = round_to_binary32(x) if x != 0 else 0
                assert oracle.fma_bits(task, it) == want, (task, it)
            x = Fraction(float(np.frombuffer(np.uint32(round_to_binary32(x * a + b)).tobytes(), np.float32)[0]))


def test_mix32_is_a_bijection_in_its_second_argument():
    for a in (0, 1, 0xdeadbeef):
        vals = {oracle.mix32(a, b) for b in range(1 << 12)}
        assert len(vals) == 1 << 12
    assert oracle.mix32(0, 0) == 0  # fmix32(0) = 0


def test_counter_body_in_topological_order():
    tr = tg.stencil_1d()
    src, dst = oracle.analyze(tr)
    rp, col = oracle.csr_from_pairs(tr.n, src, dst)
    order = largest_first_topo(tr.n, rp, col)
    st, _ = oracle.run_bodies(tr, oracle.oracle.BODY_COUNTER, state=np.zeros(16, np.int32), order=order)
    assert st.tolist() == [100] * 16
