"""rt_launch_batch32: the same launches with int32 rectangle bounds (widened on
the device). The CSR must equal the oracle's, whichever way the inputs come
(host arrays validated on the host or on the device, device arrays), also when
int32 and int64 batches are appended to one graph; bad int32 bounds are refused
by the device-side check."""
import numpy as np
import pytest

from paper_2508_16522_gb300 import grt
from paper_2508_16522_gb300 import tracegen as tg

from gpu_helpers import assert_csr_equal, ensure_built, oracle_csr

pytestmark = pytest.mark.gpu


def traces():
    return [tg.random_rects(grid=(300, 200), n=2500, rects=(1, 4), side=(1, 40), seed=31),
            tg.random_rects(grid=(5000,), n=1500, rects=(1, 3), side=(1, 300), seed=32, ndim=1),
            tg.taskbench(256, 40, "random", seed=4),
            tg.taskbench(64, 30, "stencil", seed=6, encode="explicit"),  # explicit predecessors too
            # a domain away from the origin, negative coordinates included
            tg.random_rects(grid=(90, 70), n=800, side=(1, 20), seed=33)]


def shifted(tr, off):
    """The trace moved by `off` in every dimension (domain and rectangles)."""
    o = np.full(tr.ndim, off, np.int64)
    return tg.Trace(ndim=tr.ndim, dom_lo=tr.dom_lo + o, dom_hi=tr.dom_hi + o, req_off=tr.req_off,
                    lo=tr.lo + o, hi=tr.hi + o, priv=tr.priv, pred_off=tr.pred_off, pred=tr.pred,
                    body_arg=tr.body_arg, name=tr.name + f"_shift{off}")


@pytest.mark.parametrize("how", ["host", "deferred", "device"])
def test_int32_bounds_equal_oracle(how):
    import torch
    ensure_built()
    trs = traces()
    trs[-1] = shifted(trs[-1], -1000)
    for tr in trs:
        lo32, hi32 = tr.lo.astype(np.int32), tr.hi.astype(np.int32)
        g = grt.Graph(tr.ndim, tr.dom_lo, tr.dom_hi, tile=(16, 16) if tr.ndim == 2 else (128, 1))
        arrs = [tr.req_off, lo32, hi32, tr.priv, tr.pred_off, tr.pred]
        if how == "device":
            arrs = [None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]
        g.launch(*arrs, defer_check=(how == "deferred"))
        g.analyze()
        assert_csr_equal(g, tr)
        g.close()


def test_int32_and_int64_batches_in_one_graph():
    ensure_built()
    tr = tg.random_rects(grid=(120, 100), n=1800, rects=(1, 4), side=(1, 30), seed=34)
    ref = oracle_csr(tr)
    g = grt.Graph(2, tr.dom_lo, tr.dom_hi, tile=(16, 16))
    cuts = [0, 400, 1000, 1300, tr.n]
    for k in range(len(cuts) - 1):
        a, b = cuts[k], cuts[k + 1]
        r0, r1 = tr.req_off[a], tr.req_off[b]
        ro = (tr.req_off[a:b + 1] - r0).astype(np.int32)
        lo, hi = tr.lo[r0:r1], tr.hi[r0:r1]
        if k % 2 == 0:
            lo, hi = lo.astype(np.int32), hi.astype(np.int32)
        g.launch(ro, np.ascontiguousarray(lo), np.ascontiguousarray(hi), np.ascontiguousarray(tr.priv[r0:r1]),
                 defer_check=(k == 2))
    g.analyze()
    assert_csr_equal(g, tr, ref)
    g.close()


def test_int32_bounds_outside_the_domain_refused_on_device():
    import torch
    ensure_built()
    tr = tg.taskbench(16, 4, "stencil")
    bad_hi = tr.hi.astype(np.int32)
    bad_hi[3, 0] = 99  # outside the 16-wide domain
    g = grt.Graph(2, tr.dom_lo, tr.dom_hi)
    g.launch(torch.from_numpy(tr.req_off).cuda(), torch.from_numpy(tr.lo.astype(np.int32)).cuda(),
             torch.from_numpy(bad_hi).cuda(), torch.from_numpy(tr.priv).cuda())
    with pytest.raises(grt.GrtError) as e:
        g.analyze()
    assert e.value.status == grt.RT_ERR_INVALID and "outside" in str(e.value)
    g.close()
