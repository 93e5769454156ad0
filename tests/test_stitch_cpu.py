"""Stitched replay on the CPU: the structure it relies on and its counter scheme.

A compiled graph is stitched into the surrounding program through external
pre- and post-condition vertices (Section 4.1); consecutive replays of one
trace are such a program: replay r+1 depends on replay r only through the
conditions. rt_execute_stitched runs R replays of a trace T as the DAG of T
issued R times in a row, with no barrier between replays, and relies on two
facts about that DAG under the per-cell run rule, pinned here with the
pairwise brute-force restatement of the rule (not the oracle's state machine)
and with the oracle on larger traces:

* every replay's internal edges are T's own edges;
* edges leave replay r only for replay r + 1, and the same edges (shifted) for
  every r.

Replays are not otherwise ordered: a trace whose dependences are all explicit
(the paper's Fig. 6 graph) gives replays with no edge between them, so replay
r + 2 may finish before replay r starts. The executor therefore keeps one
counter per task and replay rather than re-arming a few alternating slots; a
test below shows the alternating scheme failing on that graph. The last test
runs the executor's counter scheme itself, restated in Python, under random
interleavings of starts and completions.
"""
import random

import numpy as np

import oracle
from paper_2508_16522_gb300 import tracegen as tg

from test_oracle_pins import as_set, brute_force_edges, tiny_traces


def split_by_instance(edges, n):
    """{(a, b): {(s - a n, d - b n)}}: the edges from instance a to instance b."""
    out = {}
    for s, d in edges:
        a, b = s // n, d // n
        out.setdefault((a, b), set()).add((s - a * n, d - b * n))
    return out


def reach_from(N, edges, src):
    succ = [[] for _ in range(N)]
    for s, d in edges:
        succ[s].append(d)
    seen, stack = {src}, [src]
    while stack:
        v = stack.pop()
        for d in succ[v]:
            if d not in seen:
                seen.add(d)
                stack.append(d)
    return seen


def check_structure(T, edges_T, edges_3):
    n = T.n
    parts = split_by_instance(edges_3, n)
    for k in range(3):
        assert parts.get((k, k), set()) == edges_T, (T.name, k)
    assert not parts.get((0, 2)), T.name
    assert parts.get((0, 1), set()) == parts.get((1, 2), set()), T.name


def two_slots_suffice(n, edges_3):
    """Whether every predecessor of task v in replay 2 is reachable from v in
    replay 0 (what two alternating counter slots, re-armed at task start,
    would need)."""
    preds = {}
    for s, d in edges_3:
        preds.setdefault(d, []).append(s)
    for v in range(n):
        need = preds.get(2 * n + v, [])
        if need:
            r = reach_from(3 * n, edges_3, v)
            if not all(u in r for u in need):
                return False
    return True


def test_replays_are_not_ordered_without_shared_data():
    T = tg.fig6_fixture()  # explicit dependences only
    e3 = brute_force_edges(tg.concat([T, T, T]))
    assert not split_by_instance(e3, T.n).get((0, 1))
    assert not two_slots_suffice(T.n, e3)


def small_traces():
    out = [t for t in tiny_traces() if t.n > 0]
    for p in tg.PATTERNS:
        out.append(tg.taskbench(8, 6, p, seed=3))
        out.append(tg.taskbench(8, 6, p, seed=3, encode="explicit"))
    out.append(tg.stencil_1d(4, 5, 8))
    out.append(tg.fig6_fixture())
    return out


def test_stitching_structure_brute_force():
    for T in small_traces():
        if T.n > 40:
            continue
        T3 = tg.concat([T, T, T])
        check_structure(T, brute_force_edges(T), brute_force_edges(T3))


def test_stitching_structure_oracle_larger():
    for seed in range(6):
        T = tg.random_rects(grid=(24, 20), n=120, rects=(1, 4), side=(1, 12), seed=seed)
        e1 = as_set(*oracle.analyze(T))
        e3 = as_set(*oracle.analyze(tg.concat([T, T, T])))
        check_structure(T, e1, e3)
    for p in tg.PATTERNS:
        T = tg.taskbench(32, 12, p, seed=5)
        check_structure(T, as_set(*oracle.analyze(T)), as_set(*oracle.analyze(tg.concat([T, T, T]))))


def stitched_schedule(n, rp, col, indeg2, R, rng):
    """The stitched executor's scheme on the DAG of two instances (CSR over 2n
    tasks; targets >= n are the next replay's): one counter per task and
    replay, replay 0's starting at the in-instance in-degree and the others' at
    the full one; a decrement of a counter from 1 makes the task ready; the
    decrements replay R - 1 would send to replay R are skipped. Tasks start and
    finish in a random interleaving. Returns the (replay, task) pairs in order
    of completion, and start/finish positions."""
    indeg_in, indeg_all = indeg2[:n], indeg2[n:]
    count = [list(indeg_in)] + [list(indeg_all) for _ in range(1, R)]
    ready = [(0, v) for v in range(n) if indeg_in[v] == 0]
    ready += [(r, v) for r in range(1, R) for v in range(n) if indeg_all[v] == 0]
    running, done, t = [], [], 0
    start, finish = {}, {}
    while ready or running:
        if ready and (not running or rng.random() < 0.5):
            r, v = ready.pop(rng.randrange(len(ready)))
            assert (r, v) not in start, "a task became ready twice"
            start[(r, v)] = t
            running.append((r, v))
        else:
            r, v = running.pop(rng.randrange(len(running)))
            finish[(r, v)] = t
            done.append((r, v))
            for e in range(rp[v], rp[v + 1]):
                d = int(col[e])
                rr, dd = (r, d) if d < n else (r + 1, d - n)
                if rr >= R:
                    continue
                count[rr][dd] -= 1
                assert count[rr][dd] >= 0
                if count[rr][dd] == 0:
                    ready.append((rr, dd))
        t += 1
    return done, start, finish


def test_stitched_counter_scheme_respects_the_replayed_dag():
    rng = random.Random(7)
    cases = [tg.random_rects(grid=(16, 12), n=50, rects=(1, 4), side=(1, 8), seed=s) for s in range(4)]
    cases += [tg.taskbench(8, 5, p, seed=1) for p in tg.PATTERNS]
    cases += [tg.fig6_fixture(), tg.taskbench(8, 5, "random", seed=2, encode="explicit")]
    for T in cases:
        n, R = T.n, 5
        s2, d2 = oracle.analyze(tg.concat([T, T]))
        rp, col = oracle.csr_from_pairs(2 * n, s2, d2)
        indeg2 = np.bincount(d2, minlength=2 * n).astype(np.int64)
        sR, dR = oracle.analyze(tg.concat([T] * R))
        for trial in range(3):
            done, start, finish = stitched_schedule(n, rp, col, indeg2, R, rng)
            assert sorted(done) == [(r, v) for r in range(R) for v in range(n)], T.name
            for s, d in zip(sR.tolist(), dR.tolist()):
                a, b = (s // n, s % n), (d // n, d % n)
                assert finish[a] < start[b], (T.name, a, b)
