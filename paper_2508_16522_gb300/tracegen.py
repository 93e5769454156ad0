"""Seeded synthetic task-launch traces.

This module only *generates inputs*: streams of task launches with region
requirements (inclusive int64 rectangles plus a privilege each) and/or explicit
predecessor lists. It holds none of the dependence-analysis or execution
arithmetic, so both the CUDA path and the CPU oracle can consume its arrays.

Shapes follow the paper's Task Bench workloads (Section 6.1: a 2-D grid of
width x timesteps whose dependences run from step t-1 to step t) and the
explicit task API of Section 2.2 (``launch(p, tid, args, pre)``), at the sizes
the hot-path configurations name:

* ``stencil_1d``     16 pieces x 100 steps, 1024 cells per piece
* ``taskbench``      width 1024 x 1000 steps; stencil radius 1, butterfly
                     (partner i XOR 2^(t mod log2 width)), random fan-in 5
* ``random_rects``   4096^2 grid, 1M launches, 1-4 rects each, sides
                     log-uniform 16..1024, privileges read/write/reduce
                     60/30/10 %
* ``batch_graphs``   many independent Task Bench graphs, sizes log-uniform
* ``served_stream``  Poisson arrivals of random-rect graphs on a 1024^2 grid

Privilege codes: 0 = read, 1 = write, 2 = reduce-sum.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

READ, WRITE, REDUCE = 0, 1, 2
PATTERNS = ("stencil", "butterfly", "random")


@dataclasses.dataclass
class Trace:
    """A program-ordered stream of launches (task id = position in the stream).

    req_off : int32[n+1]   launch i owns rects [req_off[i], req_off[i+1])
    lo, hi  : int64[R, ndim] inclusive rectangle bounds
    priv    : uint8[R]
    pred_off, pred : optional explicit predecessors (ids < own id)
    body_arg: optional int32[n] per-task argument of the task body
    """

    ndim: int
    dom_lo: np.ndarray
    dom_hi: np.ndarray
    req_off: np.ndarray
    lo: np.ndarray
    hi: np.ndarray
    priv: np.ndarray
    pred_off: Optional[np.ndarray] = None
    pred: Optional[np.ndarray] = None
    body_arg: Optional[np.ndarray] = None
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.req_off.shape[0] - 1)

    @property
    def n_rects(self) -> int:
        return int(self.priv.shape[0])

    @property
    def n_cells(self) -> int:
        ext = (self.dom_hi - self.dom_lo + 1).astype(np.int64)
        return int(np.prod(ext))

    def extent(self):
        ext = (self.dom_hi - self.dom_lo + 1).astype(np.int64)
        return [int(e) for e in ext]

    def nbytes(self) -> int:
        b = self.req_off.nbytes + self.lo.nbytes + self.hi.nbytes + self.priv.nbytes
        if self.pred_off is not None:
            b += self.pred_off.nbytes + self.pred.nbytes
        if self.body_arg is not None:
            b += self.body_arg.nbytes
        return b


def _finish(ndim, dom_lo, dom_hi, counts, lo, hi, priv, pred_counts=None, pred=None,
            body_arg=None, name=""):
    req_off = np.zeros(len(counts) + 1, dtype=np.int32)
    np.cumsum(counts, out=req_off[1:])
    pred_off = None
    if pred_counts is not None:
        pred_off = np.zeros(len(pred_counts) + 1, dtype=np.int32)
        np.cumsum(pred_counts, out=pred_off[1:])
        pred = np.ascontiguousarray(pred, dtype=np.int32)
    return Trace(
        ndim=ndim,
        dom_lo=np.asarray(dom_lo, dtype=np.int64),
        dom_hi=np.asarray(dom_hi, dtype=np.int64),
        req_off=req_off,
        lo=np.ascontiguousarray(lo, dtype=np.int64).reshape(-1, ndim),
        hi=np.ascontiguousarray(hi, dtype=np.int64).reshape(-1, ndim),
        priv=np.ascontiguousarray(priv, dtype=np.uint8),
        pred_off=pred_off,
        pred=pred,
        body_arg=None if body_arg is None else np.ascontiguousarray(body_arg, dtype=np.int32),
        name=name,
    )


# ---------------------------------------------------------------------------
# 1-D stencil over pieces (16 pieces x 100 steps, 1024 cells per piece)
# ---------------------------------------------------------------------------
def stencil_1d(pieces: int = 16, steps: int = 100, piece_elems: int = 1024) -> Trace:
    """Task (i, t) has id t*pieces + i. It reads pieces i-1, i, i+1 (clipped at
    the ends, no wrap) as one read rectangle and writes piece i as a second
    rectangle. body_arg = i (the per-piece counter the body increments)."""
    n = pieces * steps
    i = np.tile(np.arange(pieces, dtype=np.int64), steps)
    lo = np.empty((n, 2), dtype=np.int64)
    hi = np.empty((n, 2), dtype=np.int64)
    lo[:, 0] = np.maximum(i - 1, 0) * piece_elems
    hi[:, 0] = (np.minimum(i + 1, pieces - 1) + 1) * piece_elems - 1
    lo[:, 1] = i * piece_elems
    hi[:, 1] = (i + 1) * piece_elems - 1
    priv = np.tile(np.array([READ, WRITE], dtype=np.uint8), n)
    return _finish(1, [0], [pieces * piece_elems - 1], np.full(n, 2), lo.reshape(-1), hi.reshape(-1),
                   priv, body_arg=i.astype(np.int32), name=f"stencil1d_{pieces}x{steps}")


# ---------------------------------------------------------------------------
# Task Bench style grids
# ---------------------------------------------------------------------------
def taskbench_preds(width: int, steps: int, pattern: str, seed: int = 0) -> np.ndarray:
    """Predecessor *columns* (indices into step t-1) of every task of steps
    1..steps-1, as an int64 [steps-1, width, k] array (k = 3 for the stencil,
    with -1 where a neighbour falls off the edge; 2 butterfly; 5 random)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cols = np.arange(width, dtype=np.int64)
    T = max(steps - 1, 0)
    if pattern == "stencil":
        left = np.where(cols > 0, cols - 1, -1)
        right = np.where(cols < width - 1, cols + 1, -1)
        one = np.stack([left, cols, right], axis=1)
        return np.broadcast_to(one, (T, width, 3)).copy()
    if pattern == "butterfly":
        logw = max(int(round(math.log2(width))), 1)
        assert (1 << logw) == width, "butterfly needs a power-of-two width"
        t = np.arange(1, steps, dtype=np.int64)
        partner = cols[None, :] ^ (np.int64(1) << (t % logw))[:, None]
        return np.stack([np.broadcast_to(cols, (T, width)), partner], axis=2)
    if pattern == "random":
        # k distinct columns of step t-1, uniform, per task (rejection: rows
        # with a repeated column are redrawn until all k are distinct)
        k = min(5, width)
        picks = rng.integers(0, width, size=(T, width, k))
        while picks.size:
            srt = np.sort(picks, axis=2)
            bad = (srt[:, :, 1:] == srt[:, :, :-1]).any(axis=2)
            nb = int(bad.sum())
            if nb == 0:
                return srt
            picks[bad] = rng.integers(0, width, size=(nb, k))
        return picks
    raise ValueError(pattern)


def taskbench(width: int = 1024, steps: int = 1000, pattern: str = "stencil", seed: int = 0,
              encode: str = "region") -> Trace:
    """Task (i, t) has id t*width + i; preds come from step t-1.

    encode='region': domain is a width x steps grid, task (i, t) writes cell
    (i, t) and reads the cells of its preds (one 1x3 read rectangle for the
    stencil, single-cell read rectangles otherwise; reads first, then the write).
    encode='explicit': no rectangles, the preds are passed as explicit lists.
    """
    n = width * steps
    pc = taskbench_preds(width, steps, pattern, seed)  # [T, w, k]
    T = pc.shape[0]
    ii = np.arange(width, dtype=np.int64)
    tt = np.arange(1, steps, dtype=np.int64)
    if encode == "explicit":
        base = ((tt - 1) * width)[:, None, None]
        valid = pc >= 0
        pcount = np.zeros(n, dtype=np.int64)
        pcount[width:] = valid.sum(axis=2).reshape(-1)
        pred = (pc + base)[valid]  # row-major: task order, then pred order
        empty = np.zeros((0,), dtype=np.int64)
        return _finish(2, [0, 0], [width - 1, steps - 1], np.zeros(n, np.int64), empty, empty,
                       np.zeros(0, dtype=np.uint8), pred_counts=pcount, pred=pred,
                       name=f"taskbench_{pattern}_{width}x{steps}_explicit")
    # region encoding: step 0 writes only; later steps read then write
    w0 = np.stack([ii, np.zeros(width, np.int64)], axis=1)
    if pattern == "stencil":
        rlo = np.stack([np.broadcast_to(np.maximum(ii - 1, 0), (T, width)),
                        np.broadcast_to(tt[:, None] - 1, (T, width))], axis=2)
        rhi = np.stack([np.broadcast_to(np.minimum(ii + 1, width - 1), (T, width)),
                        np.broadcast_to(tt[:, None] - 1, (T, width))], axis=2)
        wr = np.stack([np.broadcast_to(ii, (T, width)), np.broadcast_to(tt[:, None], (T, width))], axis=2)
        lo_t = np.stack([rlo, wr], axis=2).reshape(-1, 2)
        hi_t = np.stack([rhi, wr], axis=2).reshape(-1, 2)
        pr_t = np.tile(np.array([READ, WRITE], np.uint8), T * width)
        k = 1
    else:
        k = pc.shape[2]
        rd = np.stack([pc, np.broadcast_to((tt - 1)[:, None, None], pc.shape)], axis=3)  # [T,w,k,2]
        wr = np.stack([np.broadcast_to(ii, (T, width)), np.broadcast_to(tt[:, None], (T, width))], axis=2)
        allr = np.concatenate([rd, wr[:, :, None, :]], axis=2).reshape(-1, 2)
        lo_t = hi_t = allr
        pr_t = np.tile(np.array([READ] * k + [WRITE], np.uint8), T * width)
    lo = np.concatenate([w0, lo_t])
    hi = np.concatenate([w0, hi_t])
    counts = np.concatenate([np.ones(width, np.int64), np.full(T * width, k + 1, np.int64)])
    return _finish(2, [0, 0], [width - 1, steps - 1], counts, lo.reshape(-1), hi.reshape(-1),
                   np.concatenate([np.full(width, WRITE, np.uint8), pr_t]),
                   name=f"taskbench_{pattern}_{width}x{steps}_region")


# ---------------------------------------------------------------------------
# Random rectangles on a 2-D grid
# ---------------------------------------------------------------------------
def random_rects(grid=(4096, 4096), n: int = 1_000_000, rects=(1, 4), side=(16, 1024),
                 probs=(0.6, 0.3, 0.1), seed: int = 0, ndim: int = 2) -> Trace:
    """Each launch has a uniform number of rects in [rects[0], rects[1]]; each
    side is floor(exp(U(ln s0, ln (s1+1)))) capped at s1 (and at the grid);
    the low corner is uniform so the rect fits; privileges i.i.d. with
    ``probs`` over (read, write, reduce)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    grid = tuple(int(g) for g in (grid if ndim == 2 else grid[:1]))
    counts = rng.integers(rects[0], rects[1] + 1, size=n)
    R = int(counts.sum())
    lo = np.empty((R, ndim), np.int64)
    hi = np.empty((R, ndim), np.int64)
    for d in range(ndim):
        s = np.floor(np.exp(rng.uniform(math.log(side[0]), math.log(side[1] + 1), size=R))).astype(np.int64)
        s = np.minimum(s, min(side[1], grid[d]))
        s = np.maximum(s, 1)
        lo[:, d] = (rng.random(R) * (grid[d] - s + 1)).astype(np.int64)
        hi[:, d] = lo[:, d] + s - 1
    priv = rng.choice(3, size=R, p=list(probs)).astype(np.uint8)
    return _finish(ndim, [0] * ndim, [g - 1 for g in grid], counts, lo.reshape(-1), hi.reshape(-1),
                   priv, name=f"rand{ndim}d_{'x'.join(map(str, grid))}_n{n}_s{seed}")


# ---------------------------------------------------------------------------
# Batches of independent graphs and served request streams
# ---------------------------------------------------------------------------
def loguniform_int(rng, lo: int, hi: int, size: int) -> np.ndarray:
    return np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi + 1), size=size))).astype(np.int64).clip(lo, hi)


def batch_graph_shape(n_target: int):
    """Width 2^clamp(round(log2 N / 2), 3, 10), steps = N // width."""
    lw = int(min(max(round(math.log2(max(n_target, 2)) / 2), 3), 10))
    w = 1 << lw
    steps = max(n_target // w, 1)
    return w, steps


def batch_graph_specs(n_graphs: int = 4096, n_range=(64, 65536), seed: int = 0):
    """(width, steps, pattern, seed) of every graph of a batch: sizes
    log-uniform, patterns uniform. Any one graph can be rebuilt from its spec
    (``batch_graph``) without generating the others."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = loguniform_int(rng, n_range[0], n_range[1], n_graphs)
    pats = rng.integers(0, 3, size=n_graphs)
    out = []
    for g in range(n_graphs):
        w, steps = batch_graph_shape(int(sizes[g]))
        out.append((w, steps, PATTERNS[int(pats[g])], seed * 100003 + g))
    return out


def batch_graph(spec, encode: str = "region") -> Trace:
    w, steps, pattern, gseed = spec
    return taskbench(w, steps, pattern, seed=gseed, encode=encode)


def batch_graphs(n_graphs: int = 4096, n_range=(64, 65536), seed: int = 0,
                 encode: str = "region") -> List[Trace]:
    return [batch_graph(sp, encode) for sp in batch_graph_specs(n_graphs, n_range, seed)]


@dataclasses.dataclass
class Request:
    arrival_ns: int
    trace: Trace


def served_stream(n_requests: int = 1000, rate_per_s: float = 50_000.0, n_range=(32, 16384),
                  grid=(1024, 1024), side=(4, 256), seed: int = 0) -> List[Request]:
    """Poisson arrivals; graph sizes log-uniform; random-rect launches."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_per_s, size=n_requests)
    arr = np.cumsum(gaps)
    sizes = loguniform_int(rng, n_range[0], n_range[1], n_requests)
    out = []
    for k in range(n_requests):
        tr = random_rects(grid=grid, n=int(sizes[k]), side=side, seed=seed * 1000003 + k + 1)
        out.append(Request(int(arr[k] * 1e9), tr))
    return out


def fig6_fixture() -> Trace:
    """The four-task DAG of the paper's Fig. 6(c) (e1 -> e2, e1 -> e3,
    {e2, e3} -> e4), 0-based: 1 <- 0, 2 <- 0, 3 <- {1, 2}."""
    empty = np.zeros((0,), np.int64)
    return _finish(2, [0, 0], [0, 0], np.zeros(4, np.int64), empty, empty, np.zeros(0, np.uint8),
                   pred_counts=np.array([0, 1, 1, 2]), pred=np.array([0, 0, 1, 2]), name="fig6")


def stack_bands(traces: List[Trace], name: str = "stacked"):
    """Places 2-D traces in bands of one domain, one above the other (trace k
    moves up by the heights of the traces before it): the launches of trace k
    become tasks [off[k], off[k+1]) of the result, and no rectangle of one
    trace meets another's. Returns (trace, off)."""
    counts, los, his, pv = [], [], [], []
    y = 0
    width = 1
    off = np.zeros(len(traces) + 1, dtype=np.int32)
    for k, tr in enumerate(traces):
        assert tr.ndim == 2
        lo = tr.lo - tr.dom_lo
        hi = tr.hi - tr.dom_lo
        lo[:, 1] += y
        hi[:, 1] += y
        counts.append(np.diff(tr.req_off))
        los.append(lo)
        his.append(hi)
        pv.append(tr.priv)
        y += int(tr.dom_hi[1] - tr.dom_lo[1] + 1)
        width = max(width, int(tr.dom_hi[0] - tr.dom_lo[0] + 1))
        off[k + 1] = off[k] + tr.n
    return _finish(2, [0, 0], [width - 1, y - 1], np.concatenate(counts), np.concatenate(los).reshape(-1),
                   np.concatenate(his).reshape(-1), np.concatenate(pv), name=name), off


def concat(traces: List[Trace]) -> Trace:
    """Concatenate traces over the same domain into one program (ids shift)."""
    t0 = traces[0]
    counts = np.concatenate([np.diff(t.req_off) for t in traces])
    lo = np.concatenate([t.lo for t in traces])
    hi = np.concatenate([t.hi for t in traces])
    priv = np.concatenate([t.priv for t in traces])
    has_pred = any(t.pred_off is not None for t in traces)
    pc = pr = None
    if has_pred:
        pcs, prs, base = [], [], 0
        for t in traces:
            if t.pred_off is None:
                pcs.append(np.zeros(t.n, np.int64))
            else:
                pcs.append(np.diff(t.pred_off))
                prs.append(t.pred.astype(np.int64) + base)
            base += t.n
        pc = np.concatenate(pcs)
        pr = np.concatenate(prs) if prs else np.zeros(0, np.int64)
    ba = None
    if any(t.body_arg is not None for t in traces):
        ba = np.concatenate([t.body_arg if t.body_arg is not None else np.zeros(t.n, np.int32) for t in traces])
    return _finish(t0.ndim, t0.dom_lo, t0.dom_hi, counts, lo.reshape(-1), hi.reshape(-1), priv,
                   pred_counts=pc, pred=pr, body_arg=ba, name="+".join(t.name for t in traces))
