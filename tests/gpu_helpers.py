"""Shared helpers of the GPU tests: run a trace through libgrt and through the
oracle, and compare the canonical CSRs element by element."""
import numpy as np

import oracle
from paper_2508_16522_gb300 import build, grt
from paper_2508_16522_gb300 import tracegen as tg

_built = False


def ensure_built():
    global _built
    if not _built:
        build.build()
        grt.load()
        _built = True


def oracle_csr(tr):
    src, dst = oracle.analyze(tr)
    rp, col = oracle.csr_from_pairs(tr.n, src, dst)
    indeg = np.bincount(dst, minlength=tr.n).astype(np.int32)[:tr.n]
    return rp.astype(np.int64), col.astype(np.int32), indeg


def gpu_graph(tr, body=grt.RT_BODY_EMPTY, tile=(0, 0), spin_iters=256, flags=0, timeout_ns=0,
              device=False, defer_check=False, state_elems=None, stream=None):
    import torch
    ensure_built()
    state = out = None
    if body == grt.RT_BODY_CHECK:
        state = torch.zeros(max(tr.n_cells, 1), dtype=torch.int32, device="cuda")
    elif body == grt.RT_BODY_COUNTER:
        state = torch.zeros(state_elems or int(tr.body_arg.max()) + 1, dtype=torch.int32, device="cuda")
    if body in (grt.RT_BODY_CHECK, grt.RT_BODY_SPIN, grt.RT_BODY_FMA):
        out = torch.zeros(max(tr.n, 1), dtype=torch.int32, device="cuda")
    g = grt.Graph(tr.ndim, tr.dom_lo, tr.dom_hi, body=body, spin_iters=spin_iters, state=state, out=out,
                  tile=tile, flags=flags, timeout_ns=timeout_ns, stream=stream)
    g.launch_trace(tr, device=device, defer_check=defer_check)
    return g


def assert_csr_equal(g, tr, ref=None):
    rp_o, col_o, ind_o = ref if ref is not None else oracle_csr(tr)
    rp, col, ind = g.csr()
    assert rp.shape == rp_o.shape, (rp.shape, rp_o.shape)
    assert len(col) == len(col_o), f"{tr.name}: E gpu {len(col)} vs oracle {len(col_o)}"
    assert np.array_equal(rp.astype(np.int64), rp_o), f"{tr.name}: row_ptr differs"
    assert np.array_equal(col, col_o), f"{tr.name}: col differs"
    assert np.array_equal(ind, ind_o), f"{tr.name}: indeg differs"
    return rp, col, ind


def random_traces_small(count=24, seed0=1):
    out = []
    for k in range(count):
        s = seed0 + k
        if s % 5 == 0:
            out.append(tg.random_rects(grid=(997,), n=400, rects=(1, 4), side=(1, 90), seed=s, ndim=1))
        else:
            grid = (37 + 11 * (s % 4), 29 + 7 * (s % 3))
            out.append(tg.random_rects(grid=grid, n=300 + 40 * (s % 5), rects=(1, 4), side=(1, 17),
                                       probs=(0.5, 0.3, 0.2), seed=s))
    return out
