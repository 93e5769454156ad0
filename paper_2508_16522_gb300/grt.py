"""Thin ctypes binding of libgrt (include/grt.h).

Argument marshalling only: every step of analysis and execution runs in the
library's CUDA kernels. There is no fallback: if libgrt.so has not been built
(``paper_2508_16522_gb300.build.build()``) every call raises.

Functions keep the C names (rt_graph_create, rt_launch_batch, rt_analyze,
rt_execute, rt_replay, rt_sync, ...) and raise GrtError on a non-OK status.
``Graph`` and ``Batch`` are small conveniences that hold the handle and pass
numpy arrays (host) or torch tensors (device, or pinned host) by pointer.
"""
from __future__ import annotations

import ctypes
import os
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libgrt.so")

RT_OK, RT_ERR_INVALID, RT_ERR_OOM, RT_ERR_CUDA, RT_ERR_TIMEOUT, RT_ERR_STATE, RT_ERR_BUDGET = range(7)
STATUS_NAMES = ["RT_OK", "RT_ERR_INVALID", "RT_ERR_OOM", "RT_ERR_CUDA", "RT_ERR_TIMEOUT", "RT_ERR_STATE",
                "RT_ERR_BUDGET"]
RT_READ, RT_WRITE, RT_REDUCE_SUM = 0, 1, 2
RT_BODY_EMPTY, RT_BODY_SPIN, RT_BODY_COUNTER, RT_BODY_CHECK, RT_BODY_FMA = 0, 1, 2, 3, 4
RT_LAUNCH_HOST, RT_LAUNCH_DEVICE, RT_LAUNCH_DEFER_CHECK = 0, 1, 2
RT_GRAPH_TICKETS, RT_GRAPH_PROFILE = 1, 2
RT_EXEC_RING, RT_EXEC_OWNED = 0, 1

# every symbol include/grt.h declares (checked by the CPU tests)
EXPORTS = ["rt_graph_create", "rt_graph_destroy", "rt_graph_clear", "rt_launch_batch", "rt_launch_batch32",
           "rt_analyze", "rt_get_csr", "rt_copy_csr", "rt_graph_exec_config", "rt_execute", "rt_replay", "rt_sync",
           "rt_graph_stats", "rt_get_tickets", "rt_copy_tickets", "rt_debug_hold_task", "rt_batch_create",
           "rt_batch_execute", "rt_batch_sync", "rt_batch_counters", "rt_batch_destroy", "rt_last_error",
           "rt_device_info", "rt_kernel_launches", "rt_execute_csr_static", "rt_microbench_atomics", "rt_now_ns",
           "rt_server_create", "rt_server_submit", "rt_server_poll", "rt_server_result", "rt_server_result_state",
           "rt_server_drain", "rt_server_stats", "rt_server_destroy", "rt_tune_tile", "rt_tune_exec", "rt_tune_batch",
           "rt_batch_create_stacked", "rt_execute_events", "rt_execute_kernels", "rt_execute_stitched",
           "rt_copy_stitched_tickets", "rt_batch_capture", "rt_batch_info", "rt_graph_exec_policy",
           "rt_batch_exec_policy"]


class GrtError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")


class rt_graph_desc(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("dom_lo", ctypes.c_int64 * 2), ("dom_hi", ctypes.c_int64 * 2),
                ("body", ctypes.c_int32), ("spin_iters", ctypes.c_int32), ("state", ctypes.c_void_p),
                ("state_elems", ctypes.c_int64), ("out", ctypes.c_void_p), ("out_elems", ctypes.c_int64),
                ("stream", ctypes.c_void_p), ("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32),
                ("timeout_ns", ctypes.c_int64), ("flags", ctypes.c_int32)]


class rt_server_desc(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("dom_lo", ctypes.c_int64 * 2), ("dom_hi", ctypes.c_int64 * 2),
                ("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("body", ctypes.c_int32),
                ("spin_iters", ctypes.c_int32), ("budget_bytes", ctypes.c_int64), ("max_inflight", ctypes.c_int32),
                ("max_tasks", ctypes.c_int32), ("workers", ctypes.c_int32), ("keep_results", ctypes.c_int32),
                ("exec_blocks", ctypes.c_int32), ("exec_warps", ctypes.c_int32), ("timeout_ns", ctypes.c_int64),
                ("max_batch", ctypes.c_int32), ("reserved0", ctypes.c_int32)]


class rt_exec_config(ctypes.Structure):
    _fields_ = [("blocks", ctypes.c_int32), ("warps", ctypes.c_int32), ("claim", ctypes.c_int32),
                ("keep", ctypes.c_int32), ("ms", ctypes.c_float), ("trials", ctypes.c_int32),
                ("policy", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class rt_request_info(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int32), ("arrival_ns", ctypes.c_int64),
                ("admit_ns", ctypes.c_int64), ("posted_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64),
                ("n_tasks", ctypes.c_int64), ("n_edges", ctypes.c_int64), ("footprint_bytes", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class rt_graph_stats_t(ctypes.Structure):
    _fields_ = [("n_tasks", ctypes.c_int64), ("n_rects", ctypes.c_int64), ("n_preds", ctypes.c_int64),
                ("n_entries", ctypes.c_int64), ("n_pairs", ctypes.c_int64), ("n_edges", ctypes.c_int64),
                ("n_roots", ctypes.c_int64), ("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32),
                ("ms_analyze", ctypes.c_float), ("ms_bin", ctypes.c_float), ("ms_sort_entries", ctypes.c_float),
                ("ms_sweep", ctypes.c_float), ("ms_sort_pairs", ctypes.c_float), ("ms_csr", ctypes.c_float),
                ("ms_execute", ctypes.c_float), ("ms_exec_kernel", ctypes.c_float),
                ("exec_blocks", ctypes.c_int32), ("exec_threads", ctypes.c_int32),
                ("ms_sweep_kernel", ctypes.c_float), ("csr_by_buckets", ctypes.c_int32),
                ("pair_filter_bits", ctypes.c_int32), ("pad1", ctypes.c_int32),
                ("exec_counters", ctypes.c_int64 * 9)]

    COUNTER_NAMES = ("batches", "tasks", "edges", "claims", "cas_fail", "pushed", "idle", "slot_wait", "kept")

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "exec_counters"}
        d["exec_counters"] = dict(zip(self.COUNTER_NAMES, list(self.exec_counters)))
        return d


_lib = None


def load(path: str = LIB_PATH):
    """Loads libgrt.so; raises if it has not been built (no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libgrt.so not built at {path}: run paper_2508_16522_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {
        "rt_graph_create": [ctypes.POINTER(rt_graph_desc), ctypes.POINTER(P)],
        "rt_graph_destroy": [P],
        "rt_graph_clear": [P],
        "rt_launch_batch": [P, i32, P, P, P, P, P, P, P, i32],
        "rt_launch_batch32": [P, i32, P, P, P, P, P, P, P, i32],
        "rt_analyze": [P],
        "rt_get_csr": [P, P, P, P, P, P],
        "rt_copy_csr": [P, P, P, P],
        "rt_execute": [P],
        "rt_replay": [P, i32],
        "rt_sync": [P],
        "rt_graph_stats": [P, ctypes.POINTER(rt_graph_stats_t)],
        "rt_get_tickets": [P, P],
        "rt_copy_tickets": [P, P],
        "rt_debug_hold_task": [P, i32, i32],
        "rt_batch_create": [P, i32, P, ctypes.POINTER(P)],
        "rt_batch_execute": [P, i32, i32, i32, i32, i32],
        "rt_graph_exec_config": [P, i32, i32, i32, i32],
        "rt_batch_sync": [P, ctypes.POINTER(ctypes.c_float)],
        "rt_batch_destroy": [P],
        "rt_batch_counters": [P, ctypes.POINTER(i64), i32],
        "rt_device_info": [ctypes.POINTER(i32), ctypes.POINTER(i32)],
        "rt_kernel_launches": [ctypes.POINTER(i64)],
        "rt_execute_csr_static": [P, P, P, i32, i64, i32, P, P, P],
        "rt_microbench_atomics": [ctypes.POINTER(ctypes.c_double), i32, P],
        "rt_server_create": [ctypes.POINTER(rt_server_desc), ctypes.POINTER(P)],
        "rt_server_submit": [P, i32, P, P, P, P, i64, ctypes.POINTER(i64)],
        "rt_server_poll": [P, i64, ctypes.POINTER(rt_request_info)],
        "rt_server_result": [P, i64, P, P, P],
        "rt_server_result_state": [P, i64, P],
        "rt_server_drain": [P, i64],
        "rt_server_destroy": [P],
        "rt_server_stats": [P, ctypes.POINTER(i64), i32],
        "rt_tune_tile": [ctypes.POINTER(rt_graph_desc), i32, P, P, P, P, ctypes.c_char_p, ctypes.POINTER(i32),
                         ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_float)],
        "rt_tune_exec": [P, ctypes.c_char_p, ctypes.POINTER(rt_exec_config)],
        "rt_batch_create_stacked": [P, P, i32, P, ctypes.POINTER(P)],
        "rt_batch_capture": [ctypes.POINTER(rt_graph_desc), i32, P, P, P, P, P, P, P, i32, ctypes.POINTER(P),
                             ctypes.POINTER(P)],
        "rt_batch_info": [P, ctypes.POINTER(i64), i32],
        "rt_graph_exec_policy": [P, i32],
        "rt_batch_exec_policy": [P, i32],
        "rt_execute_events": [P, ctypes.POINTER(ctypes.c_float)],
        "rt_execute_kernels": [P, i32, i32, i32, ctypes.POINTER(ctypes.c_float)],
        "rt_execute_stitched": [P, i32, ctypes.POINTER(ctypes.c_float)],
        "rt_copy_stitched_tickets": [P, P],
        "rt_tune_batch": [P, i32, ctypes.c_char_p, ctypes.POINTER(rt_exec_config)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.rt_last_error.argtypes = []
    lib.rt_last_error.restype = ctypes.c_char_p
    lib.rt_now_ns.argtypes = []
    lib.rt_now_ns.restype = ctypes.c_int64
    _lib = lib
    return lib


def _check(st: int):
    if st != RT_OK:
        raise GrtError(st, load().rt_last_error().decode())


# ---------------------------------------------------------------------------
# C-named wrappers
# ---------------------------------------------------------------------------
def rt_graph_create(desc: rt_graph_desc) -> int:
    h = ctypes.c_void_p()
    _check(load().rt_graph_create(ctypes.byref(desc), ctypes.byref(h)))
    return h.value


def rt_graph_destroy(g):
    _check(load().rt_graph_destroy(g))


def rt_graph_clear(g):
    _check(load().rt_graph_clear(g))


def rt_launch_batch(g, n, req_off, lo, hi, priv, pred_off=None, pred=None, body_arg=None, flags=0):
    _check(load().rt_launch_batch(g, n, req_off, lo, hi, priv, pred_off, pred, body_arg, flags))


def rt_launch_batch32(g, n, req_off, lo, hi, priv, pred_off=None, pred=None, body_arg=None, flags=0):
    _check(load().rt_launch_batch32(g, n, req_off, lo, hi, priv, pred_off, pred, body_arg, flags))


def rt_analyze(g):
    _check(load().rt_analyze(g))


def rt_execute(g):
    _check(load().rt_execute(g))


def rt_replay(g, times: int):
    _check(load().rt_replay(g, times))


def rt_sync(g):
    _check(load().rt_sync(g))


def rt_graph_stats(g) -> dict:
    st = rt_graph_stats_t()
    _check(load().rt_graph_stats(g, ctypes.byref(st)))
    return st.as_dict()


def rt_debug_hold_task(g, task: int, extra: int = 1):
    _check(load().rt_debug_hold_task(g, task, extra))


def rt_device_info():
    a, b = ctypes.c_int32(), ctypes.c_int32()
    _check(load().rt_device_info(ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def rt_kernel_launches() -> int:
    c = ctypes.c_int64()
    _check(load().rt_kernel_launches(ctypes.byref(c)))
    return c.value


def rt_execute_csr_static(row_ptr, col, indeg, n_tasks: int, n_edges: int, spin_iters: int, out, tickets=None,
                          stream=None):
    """Executes a caller-held CSR (device pointers) with SPIN bodies, allocating
    nothing; `tickets` (device int32[2n], optional) receives each task's start
    and finish ticket. See include/grt.h for the limits and the sharing rule."""
    _check(load().rt_execute_csr_static(row_ptr, col, indeg, n_tasks, n_edges, spin_iters, out, tickets, stream))


def rt_microbench_atomics(stream=None) -> dict:
    """The executor's measured rooflines (see include/grt.h)."""
    out = (ctypes.c_double * 7)()
    _check(load().rt_microbench_atomics(out, 7, stream))
    names = ("dep_atomic_ns", "dep_l2_load_ns", "scatter_atomic_gops", "scatter_red_gops",
             "contended_atomic_gops", "contended_warp_agg_gops", "fma_body_ns_per_iter")
    return dict(zip(names, list(out)))


def _cache_arg(cache_path):
    return None if cache_path is None else str(cache_path).encode()


def rt_tune_tile(tr, cache_path=None, stream=None):
    """Fastest analysis tile for this trace: (tile_w, tile_h, ms)."""
    d = rt_graph_desc()
    d.ndim = tr.ndim
    for k in range(tr.ndim):
        d.dom_lo[k] = int(tr.dom_lo[k])
        d.dom_hi[k] = int(tr.dom_hi[k])
    d.stream = None if stream is None else stream.cuda_stream
    arrs = [np.ascontiguousarray(a) for a in (tr.req_off, tr.lo, tr.hi, tr.priv)]
    tw, th, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
    _check(load().rt_tune_tile(ctypes.byref(d), tr.n, *[a.ctypes.data for a in arrs], _cache_arg(cache_path),
                               ctypes.byref(tw), ctypes.byref(th), ctypes.byref(ms)))
    return tw.value, th.value, ms.value


def rt_last_error() -> str:
    return load().rt_last_error().decode()


# ---------------------------------------------------------------------------
# conveniences
# ---------------------------------------------------------------------------
def _ptr(a):
    """(pointer, is_device) of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None, False
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data, False
    # torch tensor
    assert a.is_contiguous()
    return a.data_ptr(), bool(a.is_cuda)


class Graph:
    """Holds one rt_graph and the torch buffers its body writes."""

    def __init__(self, ndim: int, dom_lo, dom_hi, body: int = RT_BODY_EMPTY, spin_iters: int = 256,
                 state=None, out=None, stream=None, tile=(0, 0), timeout_ns: int = 0, flags: int = 0):
        d = rt_graph_desc()
        d.ndim = ndim
        for k in range(ndim):
            d.dom_lo[k] = int(dom_lo[k])
            d.dom_hi[k] = int(dom_hi[k])
        d.body = body
        d.spin_iters = spin_iters
        self.state, self.out = state, out
        if state is not None:
            d.state = state.data_ptr()
            d.state_elems = state.numel()
        if out is not None:
            d.out = out.data_ptr()
            d.out_elems = out.numel()
        self.stream = stream
        d.stream = None if stream is None else stream.cuda_stream
        d.tile_w, d.tile_h = int(tile[0]), int(tile[1])
        d.timeout_ns = timeout_ns
        d.flags = flags
        self.desc = d
        self.h = rt_graph_create(d)
        self._keep = []

    def close(self):
        if self.h:
            rt_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def clear(self):
        rt_graph_clear(self.h)

    def tune(self, cache_path=None) -> dict:
        """Measures launch shapes on this analysed graph and keeps the fastest."""
        c = rt_exec_config()
        _check(load().rt_tune_exec(self.h, _cache_arg(cache_path), ctypes.byref(c)))
        return c.as_dict()

    def launch(self, req_off, lo, hi, priv, pred_off=None, pred=None, body_arg=None, defer_check=False):
        """Appends launches; numpy arrays are host pointers, CUDA tensors device pointers.
        int32 bounds go through rt_launch_batch32, int64 ones through rt_launch_batch."""
        n = int(len(req_off) - 1)
        ptrs = [_ptr(a) for a in (req_off, lo, hi, priv, pred_off, pred, body_arg)]
        dev = any(p[1] for p in ptrs)
        if dev and not all(p[1] or p[0] is None for p in ptrs):
            raise ValueError("mixing host and device arrays in one batch")
        flags = RT_LAUNCH_DEVICE if dev else (RT_LAUNCH_DEFER_CHECK if defer_check else RT_LAUNCH_HOST)
        self._keep = [req_off, lo, hi, priv, pred_off, pred, body_arg]  # alive until analyze
        widths = {str(a.dtype).split(".")[-1] for a in (lo, hi)}
        if widths == {"int32"}:
            rt_launch_batch32(self.h, n, *[p[0] for p in ptrs], flags)
        elif widths == {"int64"}:
            rt_launch_batch(self.h, n, *[p[0] for p in ptrs], flags)
        else:
            raise ValueError(f"lo and hi must both be int64 or both int32 (got {sorted(widths)})")

    def launch_trace(self, tr, device: bool = False, defer_check: bool = False):
        arrs = [tr.req_off, tr.lo, tr.hi, tr.priv, tr.pred_off, tr.pred, tr.body_arg]
        if device:
            import torch
            arrs = [None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]
        self.launch(*arrs, defer_check=defer_check)

    def analyze(self):
        rt_analyze(self.h)
        self._keep = []

    def execute(self):
        rt_execute(self.h)

    def replay(self, times: int):
        rt_replay(self.h, times)

    KERNEL_MODES = {"lifted": 0, "async": 1, "graph": 2}

    def execute_kernels(self, mode: str, iters: int = 0, threads: int = 128) -> float:
        """Every task as its own kernel (mode: lifted, async or graph); wall ms."""
        ms = ctypes.c_float()
        _check(load().rt_execute_kernels(self.h, self.KERNEL_MODES[mode], iters, threads, ctypes.byref(ms)))
        return ms.value

    def execute_stitched(self, replays: int) -> float:
        """`replays` replays of the trace this graph holds twice, joined by the
        edges between its two copies, in one launch; its time in ms."""
        ms = ctypes.c_float()
        _check(load().rt_execute_stitched(self.h, replays, ctypes.byref(ms)))
        return ms.value

    def stitched_tickets(self, replays: int):
        """(start, end) tickets of the last stitched run: int32[replays, n, 2]."""
        n = self.stats()["n_tasks"] // 2
        t = np.empty((replays, n, 2), np.int32)
        _check(load().rt_copy_stitched_tickets(self.h, t.ctypes.data))
        return t

    def execute_events(self) -> float:
        """One run through the standard, event-based executor; its kernel ms."""
        ms = ctypes.c_float()
        _check(load().rt_execute_events(self.h, ctypes.byref(ms)))
        return ms.value

    def sync(self):
        rt_sync(self.h)

    def stats(self) -> dict:
        return rt_graph_stats(self.h)

    def exec_config(self, blocks: int = 0, warps: int = 0, claim: int = 0, keep: int = 0):
        _check(load().rt_graph_exec_config(self.h, blocks, warps, claim, keep))

    def exec_policy(self, policy: int):
        _check(load().rt_graph_exec_policy(self.h, policy))

    def hold_task(self, task: int, extra: int = 1):
        rt_debug_hold_task(self.h, task, extra)

    def csr(self):
        """(row_ptr, col, indeg) copied to host numpy arrays."""
        st = self.stats()
        n, e = st["n_tasks"], st["n_edges"]
        rp = np.empty(n + 1, np.int32)
        col = np.empty(max(e, 1), np.int32)
        ind = np.empty(max(n, 1), np.int32)
        _check(load().rt_copy_csr(self.h, rp.ctypes.data, col.ctypes.data, ind.ctypes.data))
        return rp, col[:e], ind[:n]

    def tickets(self):
        n = self.stats()["n_tasks"]
        t = np.empty(2 * max(n, 1), np.int32)
        _check(load().rt_copy_tickets(self.h, t.ctypes.data))
        return t[:2 * n].reshape(n, 2)


class Batch:
    """A disjoint union of analyzed graphs run by one persistent launch."""

    def __init__(self, graphs, stream=None):
        self.graphs = list(graphs)  # the batch refers to their buffers
        arr = (ctypes.c_void_p * len(self.graphs))(*[g.h for g in self.graphs])
        h = ctypes.c_void_p()
        s = None if stream is None else stream.cuda_stream
        _check(load().rt_batch_create(arr, len(self.graphs), s, ctypes.byref(h)))
        self.h = h.value

    @classmethod
    def stacked(cls, graph, task_off, stream=None):
        """A batch of the graphs that one analysed graph holds side by side:
        tasks [task_off[k], task_off[k+1]) are graph k."""
        self = cls.__new__(cls)
        self.graphs = [graph]
        off = np.ascontiguousarray(task_off, dtype=np.int32)
        h = ctypes.c_void_p()
        s = None if stream is None else stream.cuda_stream
        _check(load().rt_batch_create_stacked(graph.h, off.ctypes.data, len(off) - 1, s, ctypes.byref(h)))
        self.h = h.value
        return self

    @classmethod
    def capture(cls, traces, body=RT_BODY_EMPTY, spin_iters=256, state=None, out=None, stream=None, tile=(0, 0),
                flags=0, inputs=None):
        """A batch of independent traces captured by ONE analysis, the library
        placing them in bands of one domain (rt_batch_capture). `inputs`
        (optional): the concatenated (req_off, lo, hi, priv) already on the
        device, as from concat_inputs(traces)."""
        ndim = traces[0].ndim
        d = rt_graph_desc()
        d.ndim = ndim
        d.body, d.spin_iters = body, spin_iters
        if state is not None:
            d.state, d.state_elems = state.data_ptr(), state.numel()
        if out is not None:
            d.out, d.out_elems = out.data_ptr(), out.numel()
        d.stream = None if stream is None else stream.cuda_stream
        d.tile_w, d.tile_h = int(tile[0]), int(tile[1])
        d.flags = flags
        task_off = np.zeros(len(traces) + 1, np.int32)
        np.cumsum([t.n for t in traces], out=task_off[1:])
        glo = np.ascontiguousarray(np.stack([t.dom_lo for t in traces]), np.int64)
        ghi = np.ascontiguousarray(np.stack([t.dom_hi for t in traces]), np.int64)
        if inputs is None:
            inputs = concat_inputs(traces)
        ptrs = [_ptr(a) for a in inputs]
        dev = any(p[1] for p in ptrs)
        h, gh = ctypes.c_void_p(), ctypes.c_void_p()
        _check(load().rt_batch_capture(ctypes.byref(d), len(traces), task_off.ctypes.data, glo.ctypes.data,
                                       ghi.ctypes.data, *[p[0] for p in ptrs], RT_LAUNCH_DEVICE if dev else 0,
                                       ctypes.byref(h), ctypes.byref(gh)))
        self = cls.__new__(cls)
        self.graphs = []
        self.h = h.value
        self.graph_h = gh.value  # owned by the batch
        self.task_off = task_off
        self._keep = (state, out, inputs)
        return self

    def info(self) -> dict:
        arr = (ctypes.c_int64 * 4)()
        _check(load().rt_batch_info(self.h, arr, 4))
        return dict(zip(("graphs", "tasks", "edges", "graph_launches"), list(arr)))

    def graph_csr(self):
        """(row_ptr, col, indeg) of the captured stacked graph (rt_batch_capture)."""
        st = rt_graph_stats(self.graph_h)
        n, e = st["n_tasks"], st["n_edges"]
        rp = np.empty(n + 1, np.int32)
        col = np.empty(max(e, 1), np.int32)
        ind = np.empty(max(n, 1), np.int32)
        _check(load().rt_copy_csr(self.graph_h, rp.ctypes.data, col.ctypes.data, ind.ctypes.data))
        return rp, col[:e], ind[:n]

    def graph_stats(self) -> dict:
        return rt_graph_stats(self.graph_h)

    def exec_policy(self, policy: int):
        """RT_EXEC_RING (default) or RT_EXEC_OWNED (the batch as one DAG, a run
        barrier between replays)."""
        _check(load().rt_batch_exec_policy(self.h, policy))

    def execute(self, replays: int = 1, blocks: int = 0, warps: int = 0, claim: int = 0, keep: int = 0):
        _check(load().rt_batch_execute(self.h, replays, blocks, warps, claim, keep))

    def sync(self) -> float:
        ms = ctypes.c_float()
        _check(load().rt_batch_sync(self.h, ctypes.byref(ms)))
        return ms.value

    def tune(self, replays: int = 1, cache_path=None) -> dict:
        """The fastest launch shape for this batch at `replays` replays; pass
        blocks/warps/claim/keep of the result to execute()."""
        c = rt_exec_config()
        _check(load().rt_tune_batch(self.h, replays, _cache_arg(cache_path), ctypes.byref(c)))
        return c.as_dict()

    def counters(self) -> dict:
        arr = (ctypes.c_int64 * 9)()
        _check(load().rt_batch_counters(self.h, arr, 9))
        return dict(zip(rt_graph_stats_t.COUNTER_NAMES, list(arr)))

    def close(self):
        if self.h:
            load().rt_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def concat_inputs(traces):
    """The launches of several traces as one (req_off, lo, hi, priv) set of host
    arrays, each trace's rectangles still in its own domain (rt_batch_capture
    places them). Concatenation only: no coordinate is changed."""
    counts = np.concatenate([np.diff(t.req_off) for t in traces])
    req_off = np.zeros(len(counts) + 1, np.int32)
    np.cumsum(counts, out=req_off[1:])
    lo = np.ascontiguousarray(np.concatenate([t.lo for t in traces]), np.int64)
    hi = np.ascontiguousarray(np.concatenate([t.hi for t in traces]), np.int64)
    priv = np.ascontiguousarray(np.concatenate([t.priv for t in traces]), np.uint8)
    return req_off, lo, hi, priv


def body_name(b: int) -> str:
    return ["EMPTY", "SPIN", "COUNTER", "CHECK", "FMA"][b]


def describe(st: dict) -> str:
    return ", ".join(f"{k}={v:.3f}" if isinstance(v, float) else f"{k}={v}" for k, v in st.items())


__all__ = [n for n in dir() if n.startswith("rt_") or n.startswith("RT_")] + [
    "Graph", "Batch", "GrtError", "load", "EXPORTS"]



def rt_now_ns() -> int:
    return int(load().rt_now_ns())


class Server:
    """Continuous-batching server: submit graphs (host arrays); worker threads
    analyse the waiting ones together (up to max_batch per analysis) and the
    persistent serving kernel runs them beside the graphs already running."""

    STATES = ("queued", "analysing", "running", "done", "failed")

    def __init__(self, ndim, dom_lo, dom_hi, body=RT_BODY_EMPTY, spin_iters=256, budget_bytes=8 << 30,
                 max_inflight=64, max_tasks=16384, workers=8, keep_results=False, tile=(0, 0),
                 exec_blocks=0, exec_warps=0, timeout_ns=0, max_batch=0):
        d = rt_server_desc()
        d.ndim = ndim
        for k in range(ndim):
            d.dom_lo[k] = int(dom_lo[k])
            d.dom_hi[k] = int(dom_hi[k])
        d.tile_w, d.tile_h = int(tile[0]), int(tile[1])
        d.body, d.spin_iters = body, spin_iters
        d.budget_bytes, d.max_inflight, d.max_tasks = budget_bytes, max_inflight, max_tasks
        d.workers, d.keep_results = workers, int(bool(keep_results))
        d.exec_blocks, d.exec_warps, d.timeout_ns = exec_blocks, exec_warps, timeout_ns
        d.max_batch = max_batch
        h = ctypes.c_void_p()
        _check(load().rt_server_create(ctypes.byref(d), ctypes.byref(h)))
        self.h = h.value

    def submit(self, tr, arrival_ns=None) -> int:
        t = ctypes.c_int64()
        arrs = [np.ascontiguousarray(a) for a in (tr.req_off, tr.lo, tr.hi, tr.priv)]
        _check(load().rt_server_submit(self.h, tr.n, *[a.ctypes.data for a in arrs],
                                       rt_now_ns() if arrival_ns is None else int(arrival_ns), ctypes.byref(t)))
        return t.value

    def poll(self, ticket) -> dict:
        info = rt_request_info()
        _check(load().rt_server_poll(self.h, ticket, ctypes.byref(info)))
        return info.as_dict()

    def result(self, ticket, n_tasks, n_edges, with_out=False):
        rp = np.empty(n_tasks + 1, np.int32)
        col = np.empty(max(n_edges, 1), np.int32)
        out = np.empty(max(n_tasks, 1), np.int32) if with_out else None
        _check(load().rt_server_result(self.h, ticket, rp.ctypes.data, col.ctypes.data,
                                       None if out is None else out.ctypes.data))
        return rp, col[:n_edges], (None if out is None else out[:n_tasks])

    def result_state(self, ticket, n_cells):
        """Final state of a finished request (CHECK body, keep_results)."""
        st = np.empty(max(n_cells, 1), np.int32)
        _check(load().rt_server_result_state(self.h, ticket, st.ctypes.data))
        return st[:n_cells]

    STAT_NAMES = ("posted", "taken", "finished", "status", "executed", "queued", "analysing", "running",
                  "kernel_running", "batches", "batched_requests", "ledger_bytes", "ledger_peak_bytes",
                  "held_bytes", "held_peak_bytes", "fixed_bytes", "trims", "budget_retries")

    def stats(self) -> dict:
        arr = (ctypes.c_int64 * len(self.STAT_NAMES))()
        _check(load().rt_server_stats(self.h, arr, len(self.STAT_NAMES)))
        return dict(zip(self.STAT_NAMES, list(arr)))

    def drain(self, timeout_ns=0):
        _check(load().rt_server_drain(self.h, timeout_ns))

    def close(self):
        if self.h:
            h, self.h = self.h, None
            _check(load().rt_server_destroy(h))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
