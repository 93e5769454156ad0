"""The batch executor's replay counters, restated in Python and run on the CPU.

A batch replays each graph R times, a graph's run r + 1 starting when its run
r has finished (its last task counted). Its counters are zeroed once per
launch and only ever incremented: a completion adds 1 to each successor's
counter, and a task of run r is ready when its counter reaches (r + 1) times
its in-degree, r travelling with the ready item. Nothing is re-armed between
runs. This is only right if run r + 1's increments of a counter never arrive
before all of run r's; they cannot, because a task of run r + 1 runs only after
run r has finished, hence after every task of run r has sent its increments.

The simulation below takes tasks and their increments in random interleavings
(several tasks in flight, increments delivered one at a time, in any order)
and checks that every (run, task) runs exactly once, in an order that respects
the DAG inside each run and the barrier between runs, with counters ending at
R times the in-degrees.
"""
import random

import numpy as np

import oracle
from paper_2508_16522_gb300 import tracegen as tg


def simulate(n, rp, col, indeg, R, rng):
    count = [0] * n
    roots = [v for v in range(n) if indeg[v] == 0]
    ready = [(0, v) for v in roots]
    inflight = []     # pending increments: (run, target)
    running = []      # started, increments not yet sent
    done_in_run = [0] * R
    order = []
    started = set()
    while ready or running or inflight:
        choice = rng.random()
        if ready and (choice < 0.4 or not (running or inflight)):
            r, v = ready.pop(rng.randrange(len(ready)))
            assert (r, v) not in started, "a task of a run became ready twice"
            started.add((r, v))
            running.append((r, v))
        elif running and (choice < 0.7 or not inflight):
            r, v = running.pop(rng.randrange(len(running)))
            order.append((r, v))
            for e in range(rp[v], rp[v + 1]):
                inflight.append((r, int(col[e])))
            done_in_run[r] += 1
            if done_in_run[r] == n and r + 1 < R:  # the run's completion seeds the next one
                ready.extend((r + 1, u) for u in roots)
        else:
            r, s = inflight.pop(rng.randrange(len(inflight)))
            old = count[s]
            count[s] += 1
            if old + 1 == (r + 1) * indeg[s]:
                ready.append((r, s))
    return order, count


def test_batch_counters_count_up_across_replays():
    rng = random.Random(11)
    cases = [tg.random_rects(grid=(16, 12), n=40, rects=(1, 4), side=(1, 8), seed=s) for s in range(4)]
    cases += [tg.taskbench(8, 5, p, seed=1) for p in tg.PATTERNS] + [tg.fig6_fixture()]
    for T in cases:
        n, R = T.n, 4
        src, dst = oracle.analyze(T)
        rp, col = oracle.csr_from_pairs(n, src, dst)
        indeg = np.bincount(dst, minlength=n).astype(np.int64)
        for trial in range(3):
            order, count = simulate(n, rp, col, indeg, R, rng)
            assert sorted(order) == [(r, v) for r in range(R) for v in range(n)], T.name
            pos = {rv: i for i, rv in enumerate(order)}
            for s, d in zip(src.tolist(), dst.tolist()):
                for r in range(R):
                    assert pos[(r, s)] < pos[(r, d)], (T.name, r, s, d)
            for r in range(1, R):  # the barrier between runs
                assert max(pos[(r - 1, v)] for v in range(n)) < min(pos[(r, v)] for v in range(n))
            assert count == [R * int(k) for k in indeg]
