"""The C ABI on a machine without a GPU: the library builds and loads, exports
every entry point include/grt.h declares, and rejects bad arguments on the host
before any CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2508_16522_gb300 import build, grt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return grt.load()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "grt.h")).read()
    return sorted(set(re.findall(r"^(?:rt_status|const char\*|int64_t)\s+(rt_\w+)\(", src, re.M)))


def test_exports_every_declared_symbol(lib):
    decl = declared_symbols()
    assert len(decl) >= 20
    assert sorted(grt.EXPORTS) == decl
    for name in decl:
        assert hasattr(lib, name), name


def desc(**kw):
    d = grt.rt_graph_desc()
    d.ndim = kw.get("ndim", 2)
    d.dom_lo[0], d.dom_lo[1] = kw.get("lo", (0, 0))
    d.dom_hi[0], d.dom_hi[1] = kw.get("hi", (63, 63))
    d.body = kw.get("body", grt.RT_BODY_EMPTY)
    d.spin_iters = kw.get("spin", 0)
    d.tile_w, d.tile_h = kw.get("tile", (0, 0))
    if "state" in kw:
        d.state = kw["state"]
        d.state_elems = kw.get("state_elems", 0)
    return d


@pytest.mark.parametrize("kw,msg", [
    (dict(ndim=3), "ndim"),
    (dict(lo=(5, 0), hi=(4, 9)), "dom_lo"),
    (dict(body=7), "body"),
    (dict(spin=-1), "spin_iters"),
    (dict(tile=(256, 16)), "tile"),
    (dict(tile=(16, 129)), "tile"),
    (dict(ndim=1, lo=(0, 0), hi=(99999, 0), tile=(2048, 1)), "1-D tile"),
    (dict(body=grt.RT_BODY_CHECK), "CHECK"),
    (dict(body=grt.RT_BODY_CHECK, state=0x1000, state_elems=10), "CHECK"),
    (dict(body=grt.RT_BODY_COUNTER), "COUNTER"),
])
def test_create_rejects(lib, kw, msg):
    with pytest.raises(grt.GrtError) as e:
        grt.rt_graph_create(desc(**kw))
    assert e.value.status == grt.RT_ERR_INVALID and msg in str(e.value)


def test_create_destroy_without_gpu(lib):
    h = grt.rt_graph_create(desc())
    grt.rt_graph_clear(h)
    with pytest.raises(grt.GrtError) as e:
        grt.rt_execute(h)
    assert e.value.status == grt.RT_ERR_STATE
    with pytest.raises(grt.GrtError) as e:
        grt.rt_replay(h, 2)
    assert e.value.status == grt.RT_ERR_STATE
    grt.rt_graph_destroy(h)


def _launch(h, req_off, lo, hi, priv, pred_off=None, pred=None, body_arg=None):
    arrs = [req_off, lo, hi, priv, pred_off, pred, body_arg]
    ptrs = [None if a is None else a.ctypes.data for a in arrs]
    entry = grt.rt_launch_batch32 if lo.dtype == np.int32 else grt.rt_launch_batch
    entry(h, len(req_off) - 1, *ptrs, grt.RT_LAUNCH_HOST)


CASES = [
    ("req_off[0]", dict(req_off=[1, 1])),
    ("decreases", dict(req_off=[0, 2, 1], lo=[[0, 0]] * 2, hi=[[1, 1]] * 2, priv=[0, 0])),
    ("lo > hi", dict(req_off=[0, 1], lo=[[3, 0]], hi=[[2, 0]], priv=[0])),
    ("outside", dict(req_off=[0, 1], lo=[[0, 0]], hi=[[64, 0]], priv=[0])),
    ("outside", dict(req_off=[0, 1], lo=[[-1, 0]], hi=[[0, 0]], priv=[0])),
    ("privilege", dict(req_off=[0, 1], lo=[[0, 0]], hi=[[0, 0]], priv=[3])),
    ("earlier task", dict(req_off=[0, 0, 0], pred_off=[0, 0, 1], pred=[1])),
    ("earlier task", dict(req_off=[0, 0], pred_off=[0, 1], pred=[-1])),
    ("pred_off", dict(req_off=[0, 0, 0, 0], pred_off=[0, 0, 1, 0], pred=[0])),
]


@pytest.mark.parametrize("width", [np.int64, np.int32])
@pytest.mark.parametrize("msg,arrs", CASES, ids=[c[0] + str(i) for i, c in enumerate(CASES)])
def test_launch_rejects_on_host(lib, msg, arrs, width):
    """rt_launch_batch (int64 bounds) and rt_launch_batch32 (int32 bounds)
    refuse the same malformed batches on the host, before any device call."""
    h = grt.rt_graph_create(desc())
    try:
        req_off = np.array(arrs["req_off"], np.int32)
        lo = np.array(arrs.get("lo", np.zeros((0, 2))), width).reshape(-1, 2)
        hi = np.array(arrs.get("hi", np.zeros((0, 2))), width).reshape(-1, 2)
        priv = np.array(arrs.get("priv", []), np.uint8)
        po = None if "pred_off" not in arrs else np.array(arrs["pred_off"], np.int32)
        pr = None if "pred" not in arrs else np.array(arrs["pred"], np.int32)
        with pytest.raises(grt.GrtError) as e:
            _launch(h, req_off, lo, hi, priv, po, pr)
        assert e.value.status == grt.RT_ERR_INVALID
        assert msg in str(e.value)
    finally:
        grt.rt_graph_destroy(h)


def test_pred_pointer_pairing(lib):
    h = grt.rt_graph_create(desc())
    try:
        ro = np.zeros(2, np.int32)
        with pytest.raises(grt.GrtError) as e:
            grt.rt_launch_batch(h, 1, ro.ctypes.data, None, None, None, ro.ctypes.data, None, None, 0)
        assert e.value.status == grt.RT_ERR_INVALID
        with pytest.raises(grt.GrtError):
            grt.rt_launch_batch(h, -1, ro.ctypes.data, None, None, None, None, None, None, 0)
        with pytest.raises(grt.GrtError):
            grt.rt_launch_batch(h, 1, ro.ctypes.data, None, None, None, None, None, None, 64)
    finally:
        grt.rt_graph_destroy(h)


def test_counter_body_needs_body_arg(lib):
    h = grt.rt_graph_create(desc(body=grt.RT_BODY_COUNTER, state=0x1000, state_elems=4))
    try:
        ro = np.zeros(2, np.int32)
        with pytest.raises(grt.GrtError) as e:
            grt.rt_launch_batch(h, 1, ro.ctypes.data, None, None, None, None, None, None, 0)
        assert "body_arg" in str(e.value)
        ba = np.array([9], np.int32)
        with pytest.raises(grt.GrtError) as e:
            grt.rt_launch_batch(h, 1, ro.ctypes.data, None, None, None, None, None, ba.ctypes.data, 0)
        assert "state buffer" in str(e.value)
    finally:
        grt.rt_graph_destroy(h)


def test_product_package_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2508_16522_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "liboracle" not in txt and "oracle.c" not in txt, f


def test_stitched_calls_refuse_before_any_gpu_work(lib):
    """rt_execute_stitched and rt_copy_stitched_tickets check their state on
    the host: no graph, an unanalysed graph, no stitched run to copy from."""
    l = grt.load()
    f = ctypes.c_float()
    assert l.rt_execute_stitched(None, 2, ctypes.byref(f)) == grt.RT_ERR_INVALID
    h = grt.rt_graph_create(desc())
    assert l.rt_execute_stitched(h, 2, ctypes.byref(f)) == grt.RT_ERR_STATE
    out = np.zeros(8, np.int32)
    assert l.rt_copy_stitched_tickets(h, None) == grt.RT_ERR_INVALID
    assert l.rt_copy_stitched_tickets(h, out.ctypes.data) == grt.RT_ERR_STATE
    grt.rt_graph_destroy(h)


def test_batch_capture_refuses_bad_arguments_without_a_gpu(lib):
    """rt_batch_capture checks its host arguments before any CUDA call."""
    import ctypes
    from paper_2508_16522_gb300 import grt
    d = grt.rt_graph_desc()
    d.ndim = 2
    out, gout = ctypes.c_void_p(), ctypes.c_void_p()
    toff = np.array([0, 2, 1], np.int32)  # decreasing
    glo = np.zeros((2, 2), np.int64)
    ghi = np.full((2, 2), 7, np.int64)
    ro = np.array([0, 1, 2], np.int32)
    lo = np.zeros((2, 2), np.int64)
    pv = np.zeros(2, np.uint8)
    args = [toff.ctypes.data, glo.ctypes.data, ghi.ctypes.data, ro.ctypes.data, lo.ctypes.data, lo.ctypes.data,
            pv.ctypes.data, 0, ctypes.byref(out), ctypes.byref(gout)]
    assert lib.rt_batch_capture(ctypes.byref(d), 2, *args) == grt.RT_ERR_INVALID
    assert b"decreases" in lib.rt_last_error()
    assert lib.rt_batch_capture(ctypes.byref(d), 0, *args) == grt.RT_ERR_INVALID
    toff2 = np.array([0, 1, 2], np.int32)
    empty_hi = np.array([[7, 7], [-1, 3]], np.int64)  # graph 1: hi < lo
    args2 = [toff2.ctypes.data, glo.ctypes.data, empty_hi.ctypes.data] + args[3:]
    assert lib.rt_batch_capture(ctypes.byref(d), 2, *args2) == grt.RT_ERR_INVALID
    assert b"empty or huge domain" in lib.rt_last_error()
    d.ndim = 3
    assert lib.rt_batch_capture(ctypes.byref(d), 2, *args) == grt.RT_ERR_INVALID
