"""Placement of independent graphs on the GPUs of one node.

Independent graphs -- the graphs of a batch, the requests of a served
stream -- share no data, so no exchange is needed between GPUs: each graph is
analysed and run whole on one device, and a graph is still launched as one
operation there (Section 4.1). What a multi-GPU job has to decide is which
device takes which graph. The work of a graph grows with its input (tasks,
region requirements, explicit predecessors; its edges follow from those), so
graphs are placed by that footprint: largest first, each on the device whose
share is smallest so far (ties to the lowest rank). A served stream cannot be
sorted before it is placed: its requests go, in arrival order, each to the
device whose share is smallest so far. Every rank computes the same placement
from the same inputs, so no message is needed to agree on it.
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np


def footprint(tr) -> int:
    """Input size of a graph: tasks + rectangles + explicit predecessors."""
    preds = 0 if tr.pred is None else int(len(tr.pred))
    return int(tr.n) + int(tr.n_rects) + preds


def assign_by_footprint(footprints: Sequence[int], world: int) -> np.ndarray:
    """owner[k] = the rank that takes graph k."""
    if world < 1:
        raise ValueError("world must be >= 1")
    fp = np.asarray(footprints, dtype=np.int64)
    owner = np.zeros(len(fp), dtype=np.int64)
    load = np.zeros(world, dtype=np.int64)
    for k in sorted(range(len(fp)), key=lambda i: (-int(fp[i]), i)):
        r = int(np.argmin(load))  # the first rank with the smallest share
        owner[k] = r
        load[r] += fp[k]
    return owner


def my_share(footprints: Sequence[int], world: int, rank: int) -> List[int]:
    """Indices of the graphs rank `rank` takes, in their original order."""
    return [int(k) for k in np.flatnonzero(assign_by_footprint(footprints, world) == rank)]


def assign_in_arrival_order(footprints: Sequence[int], world: int) -> np.ndarray:
    """owner[k] = the rank that takes request k of a stream: each request, in
    arrival order, goes to the rank whose share is smallest so far (ties to
    the lowest rank)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    fp = np.asarray(footprints, dtype=np.int64)
    owner = np.zeros(len(fp), dtype=np.int64)
    load = np.zeros(world, dtype=np.int64)
    for k in range(len(fp)):
        r = int(np.argmin(load))
        owner[k] = r
        load[r] += fp[k]
    return owner


def my_arrivals(footprints: Sequence[int], world: int, rank: int) -> List[int]:
    """Indices of the requests rank `rank` takes, in arrival order."""
    return [int(k) for k in np.flatnonzero(assign_in_arrival_order(footprints, world) == rank)]
