"""Pins the window clipping the full-size parity tests rely on, against the
oracle on whole small traces: windows that partition the domain give back
exactly the full edge set, and a task wholly inside a window keeps its exact
in- and out-edges there."""
import numpy as np

import oracle
from paper_2508_16522_gb300 import tracegen as tg
from windows import clip_to_window


def edge_set(src, dst):
    return set(zip(src.tolist(), dst.tolist()))


def window_edges(tr, wlo, whi):
    sub, ids, inside = clip_to_window(tr, wlo, whi)
    s, d = oracle.analyze(sub)
    return edge_set(ids[s], ids[d]), ids, inside


def test_partition_into_windows_gives_the_full_edge_set():
    tr = tg.random_rects(grid=(64, 48), n=400, rects=(1, 4), side=(1, 20), seed=3)
    full = edge_set(*oracle.analyze(tr))
    union = set()
    for x0, x1 in ((0, 20), (21, 63)):
        for y0, y1 in ((0, 9), (10, 30), (31, 47)):
            e, _, _ = window_edges(tr, [x0, y0], [x1, y1])
            assert e <= full
            union |= e
    assert union == full


def test_tasks_inside_a_window_keep_their_edges():
    tr = tg.random_rects(grid=(80, 80), n=500, rects=(1, 3), side=(1, 12), seed=4)
    full = edge_set(*oracle.analyze(tr))
    e, ids, inside = window_edges(tr, [10, 20], [55, 70])
    assert inside.sum() >= 20
    for t in ids[inside].tolist():
        assert {p for p in full if p[1] == t} == {p for p in e if p[1] == t}
        assert {p for p in full if p[0] == t} == {p for p in e if p[0] == t}


def test_one_dimensional_windows():
    tr = tg.random_rects(grid=(500,), n=300, rects=(1, 3), side=(1, 40), seed=5, ndim=1)
    full = edge_set(*oracle.analyze(tr))
    union = set()
    for x0, x1 in ((0, 99), (100, 377), (378, 499)):
        e, _, _ = window_edges(tr, [x0], [x1])
        union |= e
    assert union == full
