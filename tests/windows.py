"""Window clipping for parity at sizes the oracle cannot take whole.

Under the per-cell run semantics (each cell's edges depend only on the
accesses to that cell, in program order), the edges witnessed in the cells
of a window W are exactly the oracle's edges on the trace clipped to W: the
launches that touch W, in program order, each keeping its rectangles clipped
to W. So those edges must all be in the full graph, and a task whose
rectangles all lie inside W has every in- and out-edge witnessed there."""
import numpy as np

from paper_2508_16522_gb300 import tracegen as tg


def clip_to_window(tr, wlo, whi):
    """Returns (sub, ids, inside): the clipped trace, the global id of each of
    its tasks, and whether each of those tasks lies wholly inside W."""
    wlo = np.asarray(wlo, np.int64)
    whi = np.asarray(whi, np.int64)
    ilo = np.maximum(tr.lo, wlo)
    ihi = np.minimum(tr.hi, whi)
    hit = (ilo <= ihi).all(axis=1)
    within = ((tr.lo >= wlo) & (tr.hi <= whi)).all(axis=1)
    task_of = np.repeat(np.arange(tr.n), np.diff(tr.req_off))
    cnt = np.bincount(task_of[hit], minlength=tr.n)
    outside = np.bincount(task_of[~within], minlength=tr.n)
    ids = np.nonzero(cnt)[0]
    sub = tg._finish(tr.ndim, wlo, whi, cnt[ids], ilo[hit].reshape(-1), ihi[hit].reshape(-1), tr.priv[hit],
                     name=f"{tr.name}_win")
    return sub, ids, outside[ids] == 0
