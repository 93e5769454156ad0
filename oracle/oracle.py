"""ctypes wrapper around the C oracle (TEST INFRASTRUCTURE ONLY).

The C files are compiled with the host gcc into ``oracle/_lib/liboracle.so``
(``build()``; also done on first use):

* oracle.c    per-cell dependence analysis, Kahn order, sequential bodies
* interval.c  the same analysis over interval maps of run state, threaded
              over rows (for traces too large for the per-cell walk)
* alg1.c      Algorithm 1's countdown executor on host threads

All arithmetic lives in the C files; this module only marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, f) for f in ("oracle.c", "interval.c", "alg1.c")]
_LIBDIR = os.path.join(_HERE, "_lib")
_SO = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

BODY_EMPTY, BODY_SPIN, BODY_COUNTER, BODY_CHECK, BODY_FMA = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11 + pthreads, no target-specific flags)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_SO) or any(os.path.getmtime(_SO) < os.path.getmtime(s) for s in _SRCS):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", tmp] + _SRCS + ["-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load(path: str = None):
    """Loads liboracle (or, for the pin-sensitivity tests, another build of
    oracle.c at `path`)."""
    global _lib
    with _lock:
        if path is None and _lib is not None:
            return _lib
        lib = ctypes.CDLL(path or build())
        P = ctypes.c_void_p
        i32, i64, u32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
        lib.orc_analyze.restype = P
        lib.orc_analyze.argtypes = [i32, P, P, i32, P, P, P, P, P, P]
        lib.orc_result_edges.restype = i64
        lib.orc_result_edges.argtypes = [P]
        lib.orc_result_copy.restype = None
        lib.orc_result_copy.argtypes = [P, P, P]
        lib.orc_result_free.restype = None
        lib.orc_result_free.argtypes = [P]
        lib.orc_topo_order.restype = i64
        lib.orc_topo_order.argtypes = [i32, P, P, P]
        lib.orc_run.restype = i32
        lib.orc_run.argtypes = [i32, P, P, i32, P, P, P, P, P, i32, i32, P, P, P, i64]
        lib.orc_mix32.restype = u32
        lib.orc_mix32.argtypes = [u32, u32]
        lib.orc_spin.restype = u32
        lib.orc_spin.argtypes = [u32, i32]
        lib.orc_fma.restype = u32
        lib.orc_fma.argtypes = [u32, i32]
        if hasattr(lib, "orc_b3_analyze"):  # absent from a single-file build of oracle.c
            lib.orc_b3_analyze.restype = P
            lib.orc_b3_analyze.argtypes = [i32, P, P, i32, P, P, P, P, P, P, i32]
            lib.orc_b3_edges.restype = i64
            lib.orc_b3_edges.argtypes = [P]
            lib.orc_b3_copy.restype = None
            lib.orc_b3_copy.argtypes = [P, P, P]
            lib.orc_b3_free.restype = None
            lib.orc_b3_free.argtypes = [P]
            lib.orc_alg1_run.restype = i32
            lib.orc_alg1_run.argtypes = [i32, P, P, i32, i32, i32, P, P, P, P, P]
        if path is None:
            _lib = lib
        return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return None if a is None else np.ascontiguousarray(a, dtype=dt)


def analyze(tr, lib_path: str = None):
    """Edges of the trace as (src, dst) int32 arrays, sorted by (src, dst),
    deduplicated (O1 + O2 + O4)."""
    lib = _load(lib_path)
    req_off = _c(tr.req_off, np.int32)
    lo, hi = _c(tr.lo, np.int64), _c(tr.hi, np.int64)
    priv = _c(tr.priv, np.uint8)
    po, pr = _c(tr.pred_off, np.int32), _c(tr.pred, np.int32)
    dlo, dhi = _c(tr.dom_lo, np.int64), _c(tr.dom_hi, np.int64)
    h = lib.orc_analyze(tr.ndim, _p(dlo), _p(dhi), tr.n, _p(req_off), _p(lo), _p(hi), _p(priv),
                        _p(po), _p(pr))
    if not h:
        raise MemoryError("oracle analysis failed to allocate")
    try:
        e = lib.orc_result_edges(h)
        src = np.empty(e, np.int32)
        dst = np.empty(e, np.int32)
        lib.orc_result_copy(h, _p(src), _p(dst))
    finally:
        lib.orc_result_free(h)
    return src, dst


def analyze_intervals(tr, threads: int = 1, lib_path: str = None):
    """The same edges as ``analyze`` computed over interval maps of run state,
    rows split over `threads` host threads: canonical CSR (row_ptr int64[n+1],
    col int32[E])."""
    lib = _load(lib_path)
    req_off = _c(tr.req_off, np.int32)
    lo, hi = _c(tr.lo, np.int64), _c(tr.hi, np.int64)
    priv = _c(tr.priv, np.uint8)
    po, pr = _c(tr.pred_off, np.int32), _c(tr.pred, np.int32)
    dlo, dhi = _c(tr.dom_lo, np.int64), _c(tr.dom_hi, np.int64)
    h = lib.orc_b3_analyze(tr.ndim, _p(dlo), _p(dhi), tr.n, _p(req_off), _p(lo), _p(hi), _p(priv),
                           _p(po), _p(pr), int(threads))
    if not h:
        raise MemoryError("interval analysis failed to allocate")
    try:
        e = lib.orc_b3_edges(h)
        row_ptr = np.empty(tr.n + 1, np.int64)
        col = np.empty(e, np.int32)
        lib.orc_b3_copy(h, _p(row_ptr), _p(col))
    finally:
        lib.orc_b3_free(h)
    return row_ptr, col


def alg1_run(n: int, row_ptr, col, threads: int, body: int = BODY_EMPTY, spin_iters: int = 0,
             body_arg=None, state=None, tickets: bool = False):
    """Runs the CSR once with Algorithm 1's countdowns on `threads` host
    threads (bodies EMPTY, SPIN or COUNTER). Returns (state, out, tickets or
    None, ns from INIT to the last completion)."""
    lib = _load()
    rp = _c(row_ptr, np.int64)
    cl = _c(col, np.int32)
    out = np.zeros(max(n, 1), np.int32)
    st = np.ascontiguousarray(state if state is not None else np.zeros(1, np.int32), np.int32)
    ba = _c(body_arg, np.int32)
    tk = np.full(2 * max(n, 1), -1, np.int32) if tickets else None
    ns = np.zeros(1, np.int64)
    rc = lib.orc_alg1_run(n, _p(rp), _p(cl), int(threads), int(body), int(spin_iters), _p(ba), _p(st),
                          _p(out), _p(tk), _p(ns))
    if rc:
        raise MemoryError("alg1 executor failed to allocate")
    return st, out, tk, int(ns[0])


def csr_from_pairs(n: int, src: np.ndarray, dst: np.ndarray):
    """CSR by source of sorted unique pairs: (row_ptr int64[n+1], col int32[E])."""
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(src, minlength=n)[:n], out=row_ptr[1:])
    return row_ptr, np.ascontiguousarray(dst, np.int32)


def topo_order(n: int, row_ptr: np.ndarray, col: np.ndarray) -> np.ndarray:
    lib = _load()
    rp = _c(row_ptr, np.int64)
    cl = _c(col, np.int32)
    order = np.empty(max(n, 1), np.int32)
    k = lib.orc_topo_order(n, _p(rp), _p(cl), _p(order))
    if k < 0:
        raise MemoryError
    return order[:k]


def run_bodies(tr, body: int, state: np.ndarray = None, spin_iters: int = 256, order=None,
               out: np.ndarray = None):
    """Executes bodies in `order` (None = program order); returns (state, out)."""
    lib = _load()
    if state is None:
        state = np.zeros(max(tr.n_cells, 1), np.int32)
    state = np.ascontiguousarray(state, np.int32)
    if out is None:
        out = np.zeros(max(tr.n, 1), np.int32)
    ordv = None if order is None else _c(order, np.int32)
    cnt = tr.n if ordv is None else len(ordv)
    rc = lib.orc_run(tr.ndim, _p(_c(tr.dom_lo, np.int64)), _p(_c(tr.dom_hi, np.int64)), tr.n,
                     _p(_c(tr.req_off, np.int32)), _p(_c(tr.lo, np.int64)), _p(_c(tr.hi, np.int64)),
                     _p(_c(tr.priv, np.uint8)), _p(_c(tr.body_arg, np.int32)), body, spin_iters,
                     _p(state), _p(out), _p(ordv), cnt)
    if rc:
        raise MemoryError
    return state, out


def mix32(a: int, b: int) -> int:
    return int(_load().orc_mix32(a & 0xffffffff, b & 0xffffffff))


def spin(x: int, iters: int) -> int:
    return int(_load().orc_spin(x & 0xffffffff, iters))


def fma_bits(task: int, iters: int) -> int:
    """Bits of the FMA body's result for this task (binary32)."""
    return int(_load().orc_fma(task & 0xffffffff, iters))
