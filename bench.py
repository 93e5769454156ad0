"""Benchmark: tasks/s and ns/task of implicit analysis + actor-style execution.

Workload (one step): the three Task Bench graphs of width 1024 x 1000 steps
(stencil radius 1, butterfly, random fan-in 5; seed 0), each encoded as region
requirements on a 1024 x 1000 grid (a task writes its own cell and reads its
predecessors' cells), EMPTY bodies. Per graph: ingest of the launches, GPU
dependence analysis (binning, tile sweep, CSR) and one execution of the DAG.
3,072,000 tasks per step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle on the same workload (host cores).
With N > 1 (torchrun) every rank runs its own replica of the plain step (weak
scaling); the batched leg's 4096 graphs and the served leg's requests are
split across the ranks by footprint (strong scaling, no exchange between GPUs).
"""
from __future__ import annotations

import argparse
import concurrent.futures
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2508_16522_gb300 import tracegen as tg  # noqa: E402

METRIC = "tasks/sec and ns/task overhead (analysis+execution) on 1 GB300, batched vs plain"
UNIT = "tasks/s"
WIDTH, STEPS = 1024, 1000
# The autotuner picks each workload's tile and launch shapes; this file holds
# the shapes measured on this GPU model (one line per workload key), and a
# workload missing from it is tuned on the spot (a few seconds) and appended.
TUNE_CACHE = os.path.join(ROOT, "paper_2508_16522_gb300", "tune_cache.txt")
WORKLOAD = "taskbench 1024x1000 (stencil, butterfly, random fan-in 5), region-encoded, EMPTY bodies"


def load_traces(args=None):
    steps = getattr(args, "graph_steps", STEPS)
    pats = getattr(args, "patterns", ",".join(tg.PATTERNS)).split(",")
    return [tg.taskbench(WIDTH, steps, p, seed=0) for p in pats]


def config(tasks_per_step, args=None, tiles=None):
    steps = getattr(args, "graph_steps", STEPS)
    pats = getattr(args, "patterns", ",".join(tg.PATTERNS)).split(",")
    wl = WORKLOAD if (steps == STEPS and len(pats) == 3) else f"REDUCED (profiling): taskbench {WIDTH}x{steps} {pats}"
    return {"workload": wl, "patterns": pats, "width": WIDTH, "steps_per_graph": steps,
            "tasks_per_step": tasks_per_step, "tiles": tiles,
            "streams": "one stream and one host thread per graph; each graph goes through the "
                       "single-graph API (launch, analyze, execute); the input copies are issued in order "
                       "of the graphs' tuned run time, longest first, on streams whose priorities follow the "
                       "same order, then the three analyses and "
                       "executions run concurrently (each analysis blocks only its own thread)",
            "l2": "flushed between timed steps (512 MB write)", "inputs": "synthetic, seed 0"}


BATCH_GRAPHS, BATCH_REPLAYS = 4096, 20


def run_batched(grt, torch, flush, steps, world=1, rank=0):
    """The batched form: 4096 independent Task Bench graphs (sizes log-uniform
    64..65536, patterns mixed), captured once (analysis), then 20 replays of
    every graph in one persistent launch per step. With several ranks the
    graphs are split across them by footprint (shard.py; no exchange between
    GPUs): each rank captures and runs its share, and the job's time is the
    slowest rank's."""
    from paper_2508_16522_gb300 import shard
    t0 = time.perf_counter()
    all_traces = tg.batch_graphs(BATCH_GRAPHS, seed=0)
    gen_s = time.perf_counter() - t0
    share = shard.my_share([shard.footprint(t) for t in all_traces], world, rank)
    traces = [all_traces[k] for k in share]
    total_tasks = sum(t.n for t in all_traces)
    cache = TUNE_CACHE if world == 1 else None  # ranks would append to one file at once
    stream = torch.cuda.Stream()
    big = max(traces, key=lambda t: t.n)
    tile = list(grt.rt_tune_tile(big, cache)[:2])  # tuned on the largest graph
    # capture: the library places the graphs in bands of one domain and
    # analyses them ONCE (rt_batch_capture); the inputs are each graph's own
    # launches, concatenated, on the device
    inputs = [torch.from_numpy(a).cuda() for a in grt.concat_inputs(traces)]
    torch.cuda.synchronize()
    capture_ms = []
    batch = None
    for rep in range(2):  # the first capture loads and sizes everything
        if batch is not None:
            batch.close()
        t0 = time.perf_counter()
        batch = grt.Batch.capture(traces, tile=tile, stream=stream, flags=grt.RT_GRAPH_PROFILE, inputs=inputs)
        capture_ms.append((time.perf_counter() - t0) * 1e3)
    capture_ms = capture_ms[-1]
    gst = batch.graph_stats()
    ana_ms = gst["ms_analyze"]
    T = gst["n_tasks"]
    E = gst["n_edges"]
    shape = batch.tune(replays=BATCH_REPLAYS, cache_path=cache)
    launch = {k: shape[k] for k in ("blocks", "warps", "claim", "keep")}
    batch.execute(replays=BATCH_REPLAYS, **launch)
    batch.sync()
    ms = []
    for i in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(i & 255)
        batch.execute(replays=BATCH_REPLAYS, **launch)
        ms.append(batch.sync())
    kern = float(np.mean(ms))
    if world > 1:  # the job's launch and capture take as long as the slowest rank's
        kern = max_over_ranks(kern, "cuda")
        capture_ms = max_over_ranks(capture_ms, "cuda")
        T = total_tasks
    done = T * BATCH_REPLAYS
    out = {"workload": f"{BATCH_GRAPHS} Task Bench graphs, sizes log-uniform 64..65536, stencil/butterfly/random "
                       f"mixed, region-encoded, EMPTY bodies; {BATCH_REPLAYS} replays of every graph in one "
                       "persistent launch", "graphs": BATCH_GRAPHS, "tasks": T, "edges": E,
           "replays": BATCH_REPLAYS, "ms_per_launch": kern, "exec_tasks_per_s": done / (kern * 1e-3),
           "exec_ns_per_task": kern * 1e6 / done, "capture_wall_ms": capture_ms,
           "capture_ns_per_task": capture_ms * 1e6 / T, "analysis_kernel_ms": ana_ms,
           "capture": f"rt_batch_capture: the library places the graphs' launches ({sum(t.n_rects for t in traces)} "
                      f"rectangles, each graph in its own domain, inputs on the device) in bands of one domain and "
                      f"analyses them once, tile {tile}; the launch itself is relaunched from a cached CUDA graph",
           "graph_captured_launches": batch.info()["graph_launches"],
           "tasks_per_s_incl_capture": done / ((kern + capture_ms) * 1e-3), "generate_s": gen_s,
           "timed_launches": steps, "autotune": {"tile": tile, "exec": shape},
           "ranks": world, "split": "graphs placed on ranks by footprint, largest first (no exchange); time = "
                                    "slowest rank's" if world > 1 else None,
           "scaling": "strong" if world > 1 else None}
    batch.close()
    return out


SERVE_REQUESTS, SERVE_RATE = 2000, 50_000.0
SERVE_SLOTS, SERVE_WORKERS, SERVE_MAX_BATCH = 512, 4, 64
SERVE_EXEC_WARPS = 2  # serving kernel warps per SM: leaves room for 3 sweep blocks beside it


METG_ITERS = [0, 16, 64, 256, 1024, 4096, 16384, 65536]
METG_STEPS = 1000


def metg50(gran, eff):
    """Task Bench's METG(50) from a sweep of task granularities (ascending) and
    the efficiency measured at each: the granularity at which efficiency first
    reaches 1/2, interpolated linearly in efficiency and geometrically in
    granularity between the two samples that straddle it. The first
    granularity if efficiency is already 1/2 there; None if it never gets there."""
    if not gran:
        return None
    if eff[0] >= 0.5:
        return float(gran[0])
    for k in range(1, len(eff)):
        if eff[k - 1] < 0.5 <= eff[k]:
            t = (0.5 - eff[k - 1]) / (eff[k] - eff[k - 1])
            return float(np.exp(np.log(gran[k - 1]) + t * (np.log(gran[k]) - np.log(gran[k - 1]))))
    return None


def run_metg(grt, torch, ns_per_iter):
    """Task Bench's minimum effective task granularity, METG(50) (the paper's
    overhead metric, Section 6): stencil graphs of width 8 and 32, 1000 steps,
    whose task bodies run Task Bench's floating-point loop, `iters` dependent
    binary32 FMAs on one lane. Efficiency = useful time / run time, where the
    useful time of a run is steps x iters x the body's time per iteration
    measured ALONE on this GPU (one warp running nothing but the loop): one
    denominator for the box, shared by both executors, so that any time an
    executor adds to a body counts as overhead. Granularity = run time per
    step (per task on its lane); METG(50) = the granularity where efficiency
    reaches 1/2, for the compiled and the event-based executor."""
    res = {"iters": METG_ITERS, "steps": METG_STEPS,
           "body": "FMA: `iters` dependent fma.rn.f32 (x = x * 0.999f + 0.25f) on one lane per task",
           "ns_per_iteration_alone": ns_per_iter,
           "efficiency": "steps x iters x ns_per_iteration_alone / run time (one denominator per box)",
           "launch": "both executors claim one ready task per warp at a time, so that a step's long bodies "
                     "spread over warps instead of running one after another in one warp"}
    for width in (8, 32):
        tr = tg.taskbench(width, METG_STEPS, "stencil", seed=0)
        for kind in ("compiled", "events"):
            walls = []
            for it in METG_ITERS:
                out = torch.zeros(tr.n, dtype=torch.int32, device="cuda")
                g = grt.Graph(2, tr.dom_lo, tr.dom_hi, body=grt.RT_BODY_FMA, spin_iters=it, out=out,
                              flags=grt.RT_GRAPH_PROFILE)
                g.launch_trace(tr)
                g.analyze()
                g.exec_config(claim=1)  # both executors: one ready task per warp claim
                runs = []
                for _ in range(3):
                    if kind == "compiled":
                        g.execute()
                        g.sync()
                        runs.append(g.stats()["ms_exec_kernel"])
                    else:
                        runs.append(g.execute_events())
                walls.append(float(np.median(runs)))
                g.close()
            eff = [METG_STEPS * it * ns_per_iter * 1e-6 / w for it, w in zip(METG_ITERS, walls)]
            gran = [1e3 * w / METG_STEPS for w in walls]  # us per step = per task on its lane
            res[f"width{width}_{kind}"] = {"ms_per_run": [round(w, 3) for w in walls],
                                          "efficiency": [round(e, 3) for e in eff],
                                          "granularity_us": [round(x, 3) for x in gran],
                                          "metg50_us": metg50(gran, eff)}
    for width in (8, 32):
        a, b = res[f"width{width}_events"]["metg50_us"], res[f"width{width}_compiled"]["metg50_us"]
        res[f"width{width}_metg_ratio_events_over_compiled"] = round(a / b, 2) if a and b else None
    return res


def run_async_nodes(grt, torch):
    """Tasks whose bodies are whole kernels (Section 4.3): the same Task Bench
    stencil DAG (100 steps, width 8 and 32) with one 128-thread kernel per task,
    run lifted (the host launches a task once it has polled its predecessors'
    events), with async edges (every launch enqueued up front, predicated on
    events) and as one CUDA graph; the persistent executor runs the same DAG
    with its bodies in place, for context."""
    res = {"steps": 100, "threads_per_task_kernel": 128}
    for width in (8, 32):
        tr = tg.taskbench(width, 100, "stencil", seed=0)
        out = torch.zeros(tr.n, dtype=torch.int32, device="cuda")
        g = grt.Graph(2, tr.dom_lo, tr.dom_hi, body=grt.RT_BODY_SPIN, spin_iters=0, out=out,
                      flags=grt.RT_GRAPH_PROFILE)
        g.launch_trace(tr)
        g.analyze()
        for iters in (0, 4096):
            row = {}
            for mode in ("lifted", "async", "graph"):
                g.execute_kernels(mode, iters=iters, threads=128)  # warm-up (builds the CUDA graph)
                row[mode + "_ms"] = round(float(np.median([g.execute_kernels(mode, iters=iters, threads=128)
                                                           for _ in range(3)])), 3)
            row["us_per_task"] = {m: round(1e3 * row[m + "_ms"] / tr.n, 3) for m in ("lifted", "async", "graph")}
            res[f"width{width}_iters{iters}"] = row
        g.close()
    return res


def run_stitched(grt, torch):
    """Stitched replay (external pre/post-condition vertices, Section 4.1 and
    Section 5): 20 replays of a 100-step Task Bench graph of width 1024 in one
    persistent launch, once with a barrier between replays (rt_replay) and once
    joined by the edges between two copies of the trace (rt_execute_stitched),
    so that replay r + 1 starts where its own predecessors in replay r are
    done. EMPTY bodies; the barrier replay runs under the autotuner's policy and
    shape for one execution of the trace, the stitched one (a ring kernel) at the
    best of four ring shapes; times include the counter reset and seeding."""
    R = 20
    res = {"replays": R, "steps_per_replay": 100, "width": 1024,
           "launch": "barrier replay: the autotuner's policy and shape for one execution of the trace; stitched "
                     "replay (a ring kernel): the best of four ring shapes (blocks, warps, claim, keep)"}
    ring_shapes = [(304, 4, 2, 8), (304, 2, 2, 4), (152, 4, 1, 4), (152, 2, 2, 8)]
    for pat in ("stencil", "random"):
        T = tg.taskbench(1024, 100, pat, seed=0)
        g = grt.Graph(2, T.dom_lo, T.dom_hi, flags=grt.RT_GRAPH_PROFILE)
        g.launch_trace(T)
        g.analyze()
        shape = g.tune(TUNE_CACHE)
        bar = []
        for _ in range(4):
            g.replay(R)
            g.sync()
            bar.append(g.stats()["ms_execute"])
        g.close()
        g2 = grt.Graph(2, T.dom_lo, T.dom_hi, flags=grt.RT_GRAPH_PROFILE)
        g2.launch_trace(tg.concat([T, T]))
        g2.analyze()
        ana = g2.stats()["ms_analyze"]
        best = None
        for sh in ring_shapes:
            g2.exec_config(*sh)
            st = [g2.execute_stitched(R) for _ in range(4)]
            m = float(np.median(st[1:]))
            if best is None or m < best[1]:
                best = (sh, m)
        g2.close()
        b, s_ = float(np.median(bar[1:])), best[1]
        res[pat] = {"barrier_launch": {k: shape[k] for k in ("policy", "blocks", "warps", "claim", "keep")},
                    "stitched_launch": best[0], "barrier_ms": round(b, 3), "stitched_ms": round(s_, 3),
                    "speedup": round(b / s_, 2),
                    "barrier_tasks_per_s": R * T.n / (b * 1e-3), "stitched_tasks_per_s": R * T.n / (s_ * 1e-3),
                    "ms_analyze_two_copies": round(ana, 3)}
    return res


def stacked_batch(traces, max_batch, band=1024):
    """Requests as the server analyses a batch of them: request j's rectangles
    move j bands along the last dimension of a domain max_batch bands long."""
    counts, los, his = [], [], []
    for j, tr in enumerate(traces):
        lo, hi = tr.lo.copy(), tr.hi.copy()
        lo[:, 1] += j * band
        hi[:, 1] += j * band
        counts.append(np.diff(tr.req_off))
        los.append(lo)
        his.append(hi)
    return tg._finish(2, [0, 0], [band - 1, max_batch * band - 1], np.concatenate(counts),
                      np.concatenate(los).reshape(-1), np.concatenate(his).reshape(-1),
                      np.concatenate([t.priv for t in traces]), name="served_batch")


def run_served(grt, n_requests=SERVE_REQUESTS, rate=SERVE_RATE, world=1, rank=0):
    """The served form: Poisson arrivals (mean 50k graphs/s) of graphs with task
    counts log-uniform 32..16384, 1-4 rects per launch on a 1024^2 grid (sides
    log-uniform 4..256), admitted under an 8 GB device-memory budget. Requests
    are submitted when due and stamped with their due time, so submission lag
    counts as latency. With several ranks each serves its share of the stream
    (shard.py: in arrival order, each request to the rank with the smallest
    share so far), at the requests' own arrival times."""
    t0 = time.perf_counter()
    stream_all = tg.served_stream(n_requests, rate_per_s=rate, seed=0)
    reqs = stream_all
    if world > 1:
        from paper_2508_16522_gb300 import shard
        reqs = [stream_all[k] for k in shard.my_arrivals([shard.footprint(r.trace) for r in stream_all], world, rank)]
    gen_s = time.perf_counter() - t0
    # the tile is tuned on a batch of the size the stream produces (about 43)
    cache = TUNE_CACHE if world == 1 else None  # ranks would append to one file at once
    tile = list(grt.rt_tune_tile(stacked_batch([r.trace for r in stream_all[:43]], SERVE_MAX_BATCH), cache)[:2])
    srv = grt.Server(2, [0, 0], [1023, 1023], body=grt.RT_BODY_EMPTY, budget_bytes=8 << 30,
                     max_inflight=SERVE_SLOTS, max_tasks=16384, workers=SERVE_WORKERS, tile=tile,
                     max_batch=SERVE_MAX_BATCH, exec_warps=SERVE_EXEC_WARPS)
    for r in reqs[:16]:  # warm-up: grow the pool's buffers
        srv.submit(r.trace)
    srv.drain()
    base = grt.rt_now_ns() + 2_000_000
    tickets, lag = [], []
    for r in reqs:
        due = base + r.arrival_ns
        while grt.rt_now_ns() < due:
            pass
        tickets.append(srv.submit(r.trace, arrival_ns=due))
        lag.append(grt.rt_now_ns() - due)
    srv.drain()
    infos = [srv.poll(t) for t in tickets]
    sst = srv.stats()
    failed = []
    for t, i in zip(tickets, infos):
        if i["state"] != 3 and len(failed) < 3:
            try:
                srv.result(t, 0, 0)
            except grt.GrtError as e:
                failed.append(f"n={i['n_tasks']}: {e}")
    srv.close()
    if failed:
        raise RuntimeError("served requests failed: " + "; ".join(failed))
    lat = np.array([i["done_ns"] - i["arrival_ns"] for i in infos]) / 1e6
    svc = np.array([i["done_ns"] - i["admit_ns"] for i in infos]) / 1e6
    ana = np.array([i["posted_ns"] - i["admit_ns"] for i in infos]) / 1e6
    span = (max(i["done_ns"] for i in infos) - base) / 1e9
    tasks = sum(i["n_tasks"] for i in infos)
    n_requests = len(reqs)
    return {"workload": f"{n_requests} requests, Poisson arrivals at {rate:.0f} graphs/s, task counts "
                        "log-uniform 32..16384, 1-4 rects per launch on 1024^2 (sides log-uniform 4..256), "
                        f"EMPTY bodies, 8 GB budget, {SERVE_SLOTS} request slots, {SERVE_WORKERS} analysis "
                        f"workers, up to {SERVE_MAX_BATCH} waiting requests analysed together",
            "requests": n_requests, "tasks": tasks, "offered_graphs_per_s": rate,
            "achieved_graphs_per_s": n_requests / span, "tasks_per_s": tasks / span,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "service_ms": {"p50": float(np.percentile(svc, 50)), "p99": float(np.percentile(svc, 99))},
            "analysis_ms": {"p50": float(np.percentile(ana, 50)), "p99": float(np.percentile(ana, 99))},
            "mean_batch": sst["batched_requests"] / max(sst["batches"], 1), "autotune": {"tile": tile},
            "submit_lag_ms": {"p50": float(np.percentile(lag, 50)) / 1e6, "p99": float(np.percentile(lag, 99)) / 1e6},
            "generate_s": gen_s, "span_s": span}


def run_served_split(grt, world, rank, device="cuda", leg=None):
    """The served stream split across the ranks (each serves its share on its
    own GPU; no exchange): the job serves every request, in the time of its
    slowest rank. A rank whose leg fails still takes part in the reductions
    (so that no rank waits for it) and the line reports the failure. `device`
    holds the reduction tensors (the process group's); `leg` runs one rank's
    share (run_served)."""
    import torch
    import torch.distributed as dist
    err = None
    try:
        r = (leg or run_served)(grt, world=world, rank=rank)
        vals = [r["span_s"], r["latency_ms"]["p50"], r["latency_ms"]["p99"], r["analysis_ms"]["p50"]]
        sums = [float(r["requests"]), float(r["tasks"])]
    except Exception as e:  # reported below, after the reductions
        err = f"rank {rank}: {type(e).__name__}: {e}"[:300]
        vals, sums = [0.0] * 4, [0.0, 0.0]
    ok = torch.tensor([0.0 if err else 1.0], dtype=torch.float64, device=device)
    mx = torch.tensor(vals, dtype=torch.float64, device=device)
    sm = torch.tensor(sums, dtype=torch.float64, device=device)
    dist.all_reduce(ok, op=dist.ReduceOp.MIN)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    if ok.item() < 1.0:
        return {"error": err or "another rank's served leg failed", "ranks": world}
    span, p50, p99, ana = mx.tolist()
    n, tasks = sm.tolist()
    return {"workload": f"{SERVE_REQUESTS} requests, Poisson arrivals at {SERVE_RATE:.0f} graphs/s, split across "
                        f"{world} ranks", "requests": int(n), "tasks": int(tasks), "offered_graphs_per_s": SERVE_RATE,
            "achieved_graphs_per_s": n / span, "tasks_per_s": tasks / span,
            "latency_ms": {"p50": p50, "p99": p99, "note": "the largest of the ranks' percentiles"},
            "analysis_ms": {"p50": ana}, "span_s": span, "ranks": world,
            "split": "requests placed on ranks in arrival order, each on the rank with the smallest share so far "
                     "(no exchange); time = slowest rank's", "scaling": "strong"}


def run_stencil1d(grt, torch, reps=200):
    """The 1-D stencil trace (16 pieces x 100 steps = 1600 launches; task (i, t)
    reads pieces i-1..i+1 and writes piece i, 1024 cells a piece; COUNTER body,
    seed 0): the latency-bound case, where the overhead per task is all there
    is. Timed end to end through the C ABI from pinned host arrays (ingest,
    analysis, one execution and the status read-back, host clock), from inputs
    already on the device, and as a trace replay (no re-analysis)."""
    tr = tg.stencil_1d(16, 100)
    stream = torch.cuda.Stream()
    state = torch.zeros(16, dtype=torch.int32, device="cuda")
    host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in
            (tr.req_off, tr.lo, tr.hi, tr.priv, tr.body_arg)]
    dev = [a.cuda() for a in host]
    g = grt.Graph(1, tr.dom_lo, tr.dom_hi, body=grt.RT_BODY_COUNTER, state=state, stream=stream,
                  flags=grt.RT_GRAPH_PROFILE)

    def one(inp):
        g.clear()
        g.launch(*inp[:4], body_arg=inp[4])
        g.analyze()
        g.execute()
        g.sync()

    for _ in range(10):
        one(host)
    walls, ana, exe = {}, [], []
    for name, inp in (("host", host), ("device", dev)):
        w = []
        for _ in range(reps):
            t0 = time.perf_counter()
            one(inp)
            w.append(time.perf_counter() - t0)
            st = g.stats()
            ana.append(st["ms_analyze"])
            exe.append(st["ms_execute"])
        walls[name] = float(np.median(w))
    rep_w = []
    for _ in range(reps):
        t0 = time.perf_counter()
        g.replay(1)
        g.sync()
        rep_w.append(time.perf_counter() - t0)
    n, E = tr.n, g.stats()["n_edges"]
    g.close()
    us = lambda x: round(x * 1e6, 2)
    return {"workload": "1-D stencil, 16 pieces x 100 steps = 1600 launches (reads pieces i-1..i+1, writes piece "
                        "i; 1024 cells a piece), COUNTER body, one graph at a time", "tasks": n, "edges": E,
            "us_per_graph_e2e_host": us(walls["host"]), "us_per_graph_device_inputs": us(walls["device"]),
            "us_per_replay": us(float(np.median(rep_w))),
            "ns_per_task_e2e_host": round(walls["host"] * 1e9 / n, 1),
            "ns_per_task_replay": round(float(np.median(rep_w)) * 1e9 / n, 1),
            "tasks_per_s_e2e_host": n / walls["host"],
            "kernel_ms": {"analysis": round(float(np.median(ana)), 4), "execution": round(float(np.median(exe)), 4)},
            "timing": f"host clock around each call sequence, median of {reps}; the graph is 100 steps deep, "
                      "so execution is a chain of 100+ dependent wavefront steps"}


def run_rects_1m(grt, torch, flush, peaks, reps=3):
    """The implicit-analysis throughput case: 1M launches of 1-4 rectangles on a
    4096^2 grid (sides log-uniform 16..1024, read/write/reduce 60/30/10 %,
    seed 0), inputs resident on the device, analysed at the tuned tile.
    Algorithmic bytes: each launch's offset (4 B) and rectangles (2 x 2 x 8 +
    1 B each) read once, the CSR written once (row_ptr and in-degree 8 B per
    task, 4 B per edge)."""
    t0 = time.perf_counter()
    tr = tg.random_rects(grid=(4096, 4096), n=1_000_000, seed=0)
    gen_s = time.perf_counter() - t0
    tile = list(grt.rt_tune_tile(tr, TUNE_CACHE)[:2])
    stream = torch.cuda.Stream()
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (tr.req_off, tr.lo, tr.hi, tr.priv)]
    host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (tr.req_off, tr.lo, tr.hi, tr.priv)]
    g = grt.Graph(2, tr.dom_lo, tr.dom_hi, tile=tile, stream=stream, flags=grt.RT_GRAPH_PROFILE)
    runs, walls, e2e = [], [], []
    for k in range(reps + 1):  # the first run grows the buffers
        with torch.cuda.stream(stream):
            flush.fill_(k & 255)
        stream.synchronize()
        t0 = time.perf_counter()
        g.clear()
        g.launch(*dev, defer_check=True)
        g.analyze()
        stream.synchronize()
        if k:
            walls.append(time.perf_counter() - t0)
            runs.append(g.stats())
    for k in range(reps):
        with torch.cuda.stream(stream):
            flush.fill_(k & 255)
        stream.synchronize()
        t0 = time.perf_counter()
        g.clear()
        g.launch(*host, defer_check=True)
        g.analyze()
        stream.synchronize()
        e2e.append(time.perf_counter() - t0)
    g.close()
    st = runs[-1]
    n, R, E = tr.n, tr.n_rects, st["n_edges"]
    ms = float(np.median([r["ms_analyze"] for r in runs]))
    algo = 4 * n + 33 * R + 8 * n + 4 * E
    inter = 2 * 12 * st["n_entries"] + 2 * 8 * st["n_pairs"]
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    med = lambda key: round(float(np.median([r[key] for r in runs])), 3)
    return {"workload": "1M launches of 1-4 rectangles on 4096^2 (sides log-uniform 16..1024, read/write/reduce "
                        "60/30/10 %), seed 0; inputs on the device; analysis only", "tasks": n, "rects": R,
            "edges": E, "entries": st["n_entries"], "pairs": st["n_pairs"],
            "pairs_per_edge": round(st["n_pairs"] / max(E, 1), 2), "tile": tile,
            "ms_analyze": round(ms, 3), "launches_per_s": n / (ms * 1e-3), "ns_per_launch": round(ms * 1e6 / n, 2),
            "wall_ms_device_inputs": round(1e3 * float(np.median(walls)), 3),
            "wall_ms_e2e_host": round(1e3 * float(np.median(e2e)), 3),
            "phases_ms": {k: med(k) for k in ("ms_bin", "ms_sort_entries", "ms_sweep", "ms_sort_pairs", "ms_csr")},
            "hbm": {"algorithmic_bytes": algo, "intermediate_bytes": inter, "achieved_gbs": algo / (ms * 1e-3) / 1e9,
                    "peak_gbs": peak, "frac": algo / (ms * 1e-3) / 1e9 / peak},
            "generate_s": round(gen_s, 2), "timed_runs": reps,
            "l2": "flushed before each run (512 MB write)"}


# ---------------------------------------------------------------------------
# the oracle, timed on host cores (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def host_info():
    """The host the CPU numbers were taken on: core count and CPU model."""
    info = {"nproc": os.cpu_count(), "arch": os.uname().machine}
    try:
        info["affinity_cpus"] = len(os.sched_getaffinity(0))
    except Exception:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip() in ("Model name", "Vendor ID", "CPU(s)", "Thread(s) per core", "Core(s) per socket",
                             "Socket(s)", "CPU max MHz"):
                info["lscpu_" + k.strip().lower().replace(" ", "_").replace("(s)", "s")] = v.strip()
    except Exception:
        pass
    return info


def oracle_threaded_step(traces, threads):
    """The oracle on `threads` host threads: interval-map analysis (rows split
    across threads) and Algorithm 1's countdown executor (shared ready queue),
    EMPTY bodies. Returns (analysis s, execution s)."""
    import oracle
    ta = te = 0.0
    for tr in traces:
        t0 = time.perf_counter()
        rp, col = oracle.analyze_intervals(tr, threads)
        ta += time.perf_counter() - t0
        t0 = time.perf_counter()
        oracle.alg1_run(tr.n, rp, col, threads)
        te += time.perf_counter() - t0
    return ta, te


def oracle_step(traces):
    import oracle
    t0 = time.perf_counter()
    for tr in traces:
        src, dst = oracle.analyze(tr)
        rp, col = oracle.csr_from_pairs(tr.n, src, dst)
        order = oracle.topo_order(tr.n, rp, col)
        assert len(order) == tr.n
    return time.perf_counter() - t0


def run_case_served_batch(args):
    """Profiling case: the analysis of one batch of served requests (the first
    43, stacked as the server analyses them) through a plain graph, with no
    serving kernel resident, so that ncu can capture it. Not a bench line."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_16522_gb300 import grt
    reqs = tg.served_stream(SERVE_REQUESTS, rate_per_s=SERVE_RATE, seed=0)[:43]
    tr = stacked_batch([r.trace for r in reqs], SERVE_MAX_BATCH)
    tile = list(grt.rt_tune_tile(tr, TUNE_CACHE)[:2])
    stream = torch.cuda.Stream()
    g = grt.Graph(2, tr.dom_lo, tr.dom_hi, tile=tile, stream=stream, flags=grt.RT_GRAPH_PROFILE)
    inp = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (tr.req_off, tr.lo, tr.hi, tr.priv)]
    runs = []
    for k in range(args.warmup + args.steps):
        g.clear()
        g.launch(*inp)
        g.analyze()
        if k >= args.warmup:
            runs.append(g.stats())
    med = lambda key: float(np.median([r[key] for r in runs]))
    print(json.dumps({"case": "served-batch", "requests": len(reqs), "tasks": tr.n, "rects": tr.n_rects,
                      "tile": tile, "entries": runs[-1]["n_entries"], "pairs": runs[-1]["n_pairs"],
                      "edges": runs[-1]["n_edges"], "ms_analyze": med("ms_analyze"),
                      "ms_sweep_kernel": med("ms_sweep_kernel"), "ms_bin": med("ms_bin"),
                      "ms_sort_pairs": med("ms_sort_pairs"), "runs": len(runs)}), flush=True)
    g.close()
    return 0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    traces = load_traces(args)
    n_tasks = sum(t.n for t in traces)
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle_threaded_step(traces, cores)
    times = [sum(oracle_threaded_step(traces, cores)) for _ in range(args.steps)]
    total = sum(times)
    value = n_tasks * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "ns_per_task": 1e9 / value, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic", "config": config(n_tasks, args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "each step = the full workload: interval-map oracle analysis and "
                                       "Algorithm 1's countdown executor (shared ready queue), both on every "
                                       "host core", "host": host_info()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].strip().lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(value, device):
    """The largest of every rank's value (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# roofline bookkeeping
# ---------------------------------------------------------------------------
def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def kernel_source_sha(name):
    src = {"exec": "exec.cu", "sweep": "sweep.cu"}[name]
    return hashlib.sha256(open(os.path.join(ROOT, "paper_2508_16522_gb300", "csrc", src), "rb").read()).hexdigest()[:16]


def committed_traffic(name):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current source of that kernel (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(p))[name]
    except Exception:
        return None
    return d["bytes_per_launch"] if d.get("source_sha") == kernel_source_sha(name) else None


def executor_name(shapes):
    """The persistent executor kernel the graphs ran under their tuned policies."""
    pols = {int(sh.get("policy", 0)) for sh in shapes} if shapes else {0}
    if pols == {1}:
        return "k_exec_owned (persistent executor, owned chunks)"
    if pols == {0}:
        return "k_exec (persistent executor, ready ring)"
    return "k_exec_owned / k_exec (persistent executor, per-graph policy)"


def atomic_roofline_line(per_graph, mb, shapes=None):
    """The dominant kernel, the persistent executor, against the measured atomic
    roofline: algorithmic atomics per launch = E (one countdown decrement per
    edge) + 2 N / 32 (one ring reservation and one claim per 32-task warp
    batch), divided by the kernel's CUDA-event time, against the measured rate
    of scattered atomicSub on distinct addresses with the result used."""
    t_exec = sum(g["ms_exec_kernel"] for g in per_graph)
    atoms = sum(g["E"] + 2.0 * g["n"] / 32.0 for g in per_graph)
    launches = len(per_graph)
    achieved = (atoms / launches) / (t_exec / launches * 1e-3) / 1e9
    peak = mb["scatter_atomic_gops"]
    return {"kernel": executor_name(shapes), "bound": "atomic", "achieved": achieved, "peak": peak,
            "unit": "Gatomic/s", "frac": achieved / peak, "traffic": committed_traffic("exec"),
            "traffic_unit": "DRAM bytes per launch (ncu)",
            "algorithmic_atomics_per_launch": atoms / launches, "avg_launch_ms": t_exec / launches,
            "peak_source": "measured in this run: scattered int32 atomicSub on distinct addresses, result used "
                           "(rt_microbench_atomics)", "share_of_step": None}


def roofline(per_graph, peaks, shapes=None):
    """per_graph: list of dicts (n, E, entries, pairs, ms_exec_kernel, ms_sweep_kernel) averaged
    over the timed steps. Algorithmic bytes:
      executor: 16 B per task (row_ptr pair, indeg read, counter re-arm) + 12 B per edge
                (col read, counter read-modify-write)
      sweep:    8 B per binned entry read + 8 B per candidate pair written."""
    t_exec = sum(g["ms_exec_kernel"] for g in per_graph)
    t_sweep = sum(g["ms_sweep_kernel"] for g in per_graph)
    if t_exec >= t_sweep:
        name, ms = "exec", t_exec
        algo = sum(16 * g["n"] + 12 * g["E"] for g in per_graph)
    else:
        name, ms = "sweep", t_sweep
        algo = sum(8 * g["entries"] + 8 * g["pairs"] for g in per_graph)
    launches = len(per_graph)
    achieved = (algo / launches) / (ms / launches * 1e-3) / 1e9
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    traffic = committed_traffic(name)
    return {"kernel": {"exec": executor_name(shapes), "sweep": "k_sweep (tile interference sweep)"}[name],
            "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "algorithmic_bytes_per_launch": algo / launches,
            "avg_launch_ms": ms / launches, "peak_source": "measured" if peaks else "fallback",
            "share_of_step": None}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_16522_gb300 import grt

    traces = load_traces(args)
    n_tasks = sum(t.n for t in traces)
    # one stream per graph: the graphs of a step are independent, so one
    # graph's analysis runs while another's persistent executor does
    streams = [torch.cuda.Stream() for _ in traces]
    stream = streams[0]
    dev_inputs = [[torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (t.req_off, t.lo, t.hi, t.priv)]
                  for t in traces]
    # end-to-end inputs: pinned host arrays, the bounds as int32 where they fit
    # (rt_launch_batch32 widens them on the device: half the coordinate bytes
    # on the host link)
    i32 = np.iinfo(np.int32)
    coord32 = all(t.lo.min() >= i32.min and t.hi.max() <= i32.max for t in traces)
    host_inputs = [[torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
                    for a in (t.req_off, t.lo.astype(np.int32) if coord32 else t.lo,
                              t.hi.astype(np.int32) if coord32 else t.hi, t.priv)]
                   for t in traces]
    tiles = [list(grt.rt_tune_tile(t, TUNE_CACHE)[:2]) for t in traces]
    graphs = [grt.Graph(2, t.dom_lo, t.dom_hi, tile=tl, stream=st, flags=grt.RT_GRAPH_PROFILE)
              for t, tl, st in zip(traces, tiles, streams)]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    order = list(range(len(graphs)))
    # one host thread per graph: rt_analyze blocks its caller while it sizes
    # buffers, so the graphs' analyses overlap only when their threads call
    # them together (the library allows calls on distinct graphs from distinct
    # threads; ctypes releases the interpreter lock for each call)
    from concurrent.futures import ThreadPoolExecutor
    pool = ThreadPoolExecutor(max_workers=len(graphs), initializer=torch.cuda.set_device, initargs=(local,))

    def analyze_execute(i):
        graphs[i].analyze()
        graphs[i].execute()  # asynchronous
    copy_done = [torch.cuda.Event() for _ in graphs]

    def step(inputs, defer=False, overlap=True):
        if not overlap:  # one graph after another
            for g, inp in zip(graphs, inputs):
                g.clear()
                g.launch(*inp, defer_check=defer)
                g.analyze()
                g.execute()
                g.sync()
            return
        # longest execution first (the autotuner's measured run time), so that
        # the step's tail is as short as the overlap allows
        prev = None
        for i in order:
            graphs[i].clear()
            if defer and prev is not None:
                # host inputs: one graph's copies after the other's, in the
                # order of the step, so the first graph's analysis starts as
                # soon as its own inputs are in (concurrent copies would share
                # the link and all finish late)
                streams[i].wait_event(prev)
            graphs[i].launch(*inputs[i], defer_check=defer)  # copies in, asynchronous
            if defer:
                prev = copy_done[i]
                prev.record(streams[i])
        list(pool.map(analyze_execute, order))
        for g in graphs:
            g.sync()

    def stats():
        out = []
        for g in graphs:
            s = g.stats()
            out.append({"n": s["n_tasks"], "E": s["n_edges"], "entries": s["n_entries"], "pairs": s["n_pairs"],
                        "ms_exec_kernel": s["ms_exec_kernel"], "ms_sweep_kernel": s["ms_sweep_kernel"],
                        "ms_analyze": s["ms_analyze"], "ms_bin": s["ms_bin"],
                        "ms_sort_entries": s["ms_sort_entries"], "ms_sweep": s["ms_sweep"],
                        "ms_sort_pairs": s["ms_sort_pairs"], "ms_csr": s["ms_csr"], "ms_execute": s["ms_execute"]})
        return out

    def timed(inputs, k, defer=False, overlap=True):
        """CUDA events on the first graph's stream; the other streams start
        after its start event and it waits for theirs before its end event."""
        ms, per = [], []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        done = [torch.cuda.Event() for _ in streams]
        for i in range(k):
            with torch.cuda.stream(stream):
                flush.fill_(i & 255)
            e0.record(stream)
            for st in streams[1:]:
                st.wait_event(e0)
            step(inputs, defer, overlap)
            for st, ev in zip(streams[1:], done[1:]):
                ev.record(st)
                stream.wait_event(ev)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            per.append(stats())
        return ms, per

    for _ in range(args.warmup):
        step(dev_inputs)
    exec_shapes = [g.tune(TUNE_CACHE) for g in graphs]  # outside the timed region
    order[:] = sorted(range(len(graphs)), key=lambda i: -exec_shapes[i]["ms"])
    # stream priorities in the same order: when the graphs' analyses compete for
    # the SMs, the blocks of the graph with the longest execution are scheduled
    # first, so its executor starts earliest. A graph keeps the stream it was
    # created on, so the graphs are made again on prioritised streams (same
    # tiles; their launch shapes come back from the tuner's cache)
    least, greatest = torch.cuda.Stream.priority_range()
    prio = [0] * len(graphs)
    for r, i in enumerate(order):
        prio[i] = min(least, greatest + r) if greatest < least else least
    for g in graphs:
        g.close()
    streams[:] = [torch.cuda.Stream(priority=p) for p in prio]
    stream = streams[0]
    graphs[:] = [grt.Graph(2, t.dom_lo, t.dom_hi, tile=tl, stream=st, flags=grt.RT_GRAPH_PROFILE)
                 for t, tl, st in zip(traces, tiles, streams)]
    for _ in range(args.warmup):
        step(dev_inputs)
    exec_shapes = [g.tune(TUNE_CACHE) for g in graphs]
    step(dev_inputs)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = grt.rt_kernel_launches()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ms, per = timed(dev_inputs, args.steps)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    launches = grt.rt_kernel_launches() - l0
    clk = clocks.stop()
    total_ms = sum(ms)
    if world > 1:
        total_ms = max_over_ranks(total_ms, "cuda")
        dist.barrier()

    # the same graphs one after another on their streams (no overlap), for reference
    seq_ms, _ = timed(dev_inputs, args.steps, overlap=False)

    # end to end through the host API: pinned host arrays, H2D inside the step
    e2e_ms = [float("nan")]
    if not args.no_e2e:
        for _ in range(max(1, args.warmup // 2)):
            step(host_inputs, defer=True)
        e2e_ms, _ = timed(host_inputs, args.steps, defer=True)
    h2d = sum(sum(int(a.numel() * a.element_size()) for a in inp) for inp in host_inputs)
    # the host link alone: one pinned-to-device copy of a step's input bytes
    # (the end-to-end step cannot beat it: its copies sit on the same link)
    link_gbs = None
    if not args.no_e2e:
        src = torch.empty(h2d, dtype=torch.uint8).pin_memory()
        dst = torch.empty(h2d, dtype=torch.uint8, device="cuda")
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        best = float("inf")
        for _ in range(4):
            with torch.cuda.stream(stream):
                c0.record(stream)
                dst.copy_(src, non_blocking=True)
                c1.record(stream)
            c1.synchronize()
            best = min(best, c0.elapsed_time(c1))
        link_gbs = h2d / (best * 1e-3) / 1e9
        del src, dst
    batched = None
    if not args.no_batched:
        batched = run_batched(grt, torch, flush, max(1, min(args.steps, 3)), world, rank)
    # the executor's own rooflines (dependent atomic latency, scattered atomics)
    # and the FMA body's rate alone
    mb = grt.rt_microbench_atomics()
    metg = None
    if world == 1 and not args.no_metg:
        metg = run_metg(grt, torch, mb["fma_body_ns_per_iter"])
    async_nodes = stitched = None
    if world == 1 and not args.no_extras:
        async_nodes = run_async_nodes(grt, torch)
        stitched = run_stitched(grt, torch)
    served = None
    if world > 1 and not args.no_served:
        served = run_served_split(grt, world, rank)
    if world == 1 and not args.no_served:
        served = run_served(grt)
        # the same stream offered at 3/4 of the rate just achieved: latency
        # without the queue that an offered load beyond capacity builds up
        calm = run_served(grt, rate=0.75 * served["achieved_graphs_per_s"])
        served["at_three_quarters_of_capacity"] = {
            k: calm[k] for k in ("offered_graphs_per_s", "achieved_graphs_per_s", "tasks_per_s", "latency_ms",
                                 "service_ms", "analysis_ms", "mean_batch")}

    value = world * n_tasks * args.steps / (total_ms * 1e-3)
    e2e_value = None if args.no_e2e else n_tasks * args.steps / (sum(e2e_ms) * 1e-3)
    avg = [{k: float(np.mean([p[i][k] for p in per])) for k in per[0][i]} for i in range(len(graphs))]
    # the same graphs with 256-iteration integer spin bodies (the Task Bench
    # workload's second body), execution only: the body adds a chain of 256 dependent multiply-adds
    # to every wavefront step
    spin = events = None
    if world == 1 and not args.no_extras:
        spin_ms = []
        for t, tl, st_ in zip(traces, tiles, streams):
            out = torch.zeros(t.n, dtype=torch.int32, device="cuda")
            gs = grt.Graph(2, t.dom_lo, t.dom_hi, body=grt.RT_BODY_SPIN, spin_iters=256, out=out, tile=tl,
                           stream=st_, flags=grt.RT_GRAPH_PROFILE)
            gs.launch_trace(t, defer_check=True)
            gs.analyze()
            gs.tune(TUNE_CACHE)
            runs = []
            for _ in range(4):
                gs.execute()
                gs.sync()
                runs.append(gs.stats()["ms_exec_kernel"])
            spin_ms.append(float(np.median(runs[1:])))
            gs.close()
        empty_ms = []  # the EMPTY graphs run alone too (the timed step overlaps them)
        for g in graphs:
            runs = []
            for _ in range(4):
                g.execute()
                g.sync()
                runs.append(g.stats()["ms_exec_kernel"])
            empty_ms.append(float(np.median(runs[1:])))
        # the same graphs through the standard, event-based executor (fresh
        # events and waiter lists built at every run) against the compiled one
        ev_ms = []
        for g in graphs:
            runs = [g.execute_events() for _ in range(4)]
            ev_ms.append(float(np.median(runs[1:])))
        events = {"ms_kernel_event_based": ev_ms, "ms_kernel_compiled": empty_ms,
                  "ratio": [round(a / b, 2) for a, b in zip(ev_ms, empty_ms)],
                  "event_based_tasks_per_s": n_tasks / (sum(ev_ms) * 1e-3),
                  "compiled_tasks_per_s": n_tasks / (sum(empty_ms) * 1e-3),
                  "note": "EMPTY bodies, each graph alone; the paper reports 1.7-5.3x lower overheads for its "
                          "compiled form in Realm (CPU clusters), quoted as context"}
        spin = {"body": "SPIN, 256 iterations of an int32 LCG per task", "ms_exec_kernel": spin_ms,
                "ms_exec_kernel_empty_alone": empty_ms,
                "exec_tasks_per_s": n_tasks / (sum(spin_ms) * 1e-3),
                "added_ns_per_wavefront_step": [round(1e6 * (a - b) / STEPS, 1) for a, b in zip(spin_ms, empty_ms)],
                "note": "each of the 1000 wavefront steps carries one 256-long chain of dependent integer "
                        "multiply-adds on its critical path"}

    peaks = measured_peaks()
    roof_hbm = roofline(avg, peaks, exec_shapes)
    roof = atomic_roofline_line(avg, mb, exec_shapes)
    # executor kernel time over step time; above 1 when the graphs' executions overlap
    for r in (roof, roof_hbm):
        r["share_of_step"] = (r["avg_launch_ms"] * len(graphs)) / (total_ms / args.steps) if world == 1 else None
    stencil1d = rects_1m = None
    if world == 1 and not args.no_extras:
        stencil1d = run_stencil1d(grt, torch)
        rects_1m = run_rects_1m(grt, torch, flush, peaks)
    # the analysis against HBM: algorithmic bytes are the launches and
    # rectangles read once and the CSR written once (req_off 4 B per task,
    # 2 x ndim x 8 + 1 B per rectangle; row_ptr and indeg 8 B per task, col
    # 4 B per edge); the intermediate traffic (binned entries, candidate pairs,
    # both sorted) is reported beside it
    R_per = [float(t.n_rects) for t in traces]
    ana_alg = [4 * a["n"] + 33 * r + 8 * a["n"] + 4 * a["E"] for a, r in zip(avg, R_per)]
    ana_inter = [2 * 12 * a["entries"] + 2 * 8 * a["pairs"] for a in avg]
    ana_ms_tot = sum(a["ms_analyze"] for a in avg)
    analysis_roof = {
        "bound": "hbm", "unit": "GB/s", "peak": peaks["hbm_gbs"] if peaks else 6800.0,
        "algorithmic_bytes_per_step": sum(ana_alg), "intermediate_bytes_per_step": sum(ana_inter),
        "ms_per_step": ana_ms_tot,
        "achieved": sum(ana_alg) / (ana_ms_tot * 1e-3) / 1e9,
        "note": "a dozen dependent phases (bin, sort, sweep, sort, CSR) with host syncs between them; the "
                "intermediate bytes (entries and pairs written and sorted) dwarf the algorithmic ones"}
    analysis_roof["frac"] = analysis_roof["achieved"] / analysis_roof["peak"]
    ex_ms = sum(a["ms_exec_kernel"] for a in avg)
    edges = sum(a["E"] for a in avg)
    depth = getattr(args, "graph_steps", STEPS)
    step_ns = [1e6 * a["ms_exec_kernel"] / depth for a in avg]
    atomic_roof = {
        "measured": {k: round(v, 4) for k, v in mb.items()},
        "exec_edge_decrements_gops": edges / (ex_ms * 1e-3) / 1e9,
        "frac_of_scatter_atomic_throughput": edges / (ex_ms * 1e-3) / 1e9 / mb["scatter_atomic_gops"],
        "ns_per_wavefront_step": [round(x, 1) for x in step_ns],
        "dep_atomic_latencies_per_step": [round(x / mb["dep_atomic_ns"], 2) for x in step_ns],
        "note": "each graph is 1000 dependent steps deep; a step cannot take less than one dependent atomic "
                "round trip, so dep_atomic_latencies_per_step is the executor's distance from its latency floor"}

    line = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cores = os.cpu_count() or 1
            ta, te = oracle_threaded_step(traces, cores)
            t1a, t1e = oracle_threaded_step(traces, 1)
            secs = oracle_step(traces)
            cpu = {"value": n_tasks / (ta + te), "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": "one pass of the full workload (3 graphs, 3.07M tasks, EMPTY bodies): interval-map "
                             "oracle analysis (rows split over every host core) + Algorithm 1's countdown "
                             "executor (atomic countdowns, one shared ready queue, every host core)",
                   "analysis_s": round(ta, 3), "execution_s": round(te, 3),
                   "analysis_tasks_per_s": n_tasks / ta, "execution_tasks_per_s": n_tasks / te,
                   "one_thread": {"analysis_s": round(t1a, 3), "execution_s": round(t1e, 3),
                                  "value": n_tasks / (t1a + t1e)},
                   "per_cell_oracle_one_thread": {"value": n_tasks / secs, "seconds": round(secs, 3),
                                                  "what": "per-cell oracle analysis + Kahn order"},
                   "note": "with EMPTY bodies the threaded executor is slower than one thread: every decrement "
                           "moves a counter's cache line between cores",
                   "host": host_info()}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "ns_per_task": 1e9 / value * world,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
                "data": "synthetic", "config": config(n_tasks, args, tiles), "form": "plain",
                "autotune": {"tiles": tiles, "exec": exec_shapes, "cache": os.path.relpath(TUNE_CACHE, ROOT)},
                "e2e": None if args.no_e2e else {
                    "value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": 8 * len(graphs), "ms_per_step": sum(e2e_ms) / args.steps,
                    "validation": "on the device (RT_LAUNCH_DEFER_CHECK)",
                    "coordinates": "int32 (rt_launch_batch32)" if coord32 else "int64 (rt_launch_batch)",
                    "h2d_link_gbs": link_gbs,
                    "h2d_copy_ms_per_step": h2d / (link_gbs * 1e9) * 1e3 if link_gbs else None,
                    "note": "the step's input copies run one graph after another on the host link; "
                            "h2d_copy_ms_per_step is their time alone at the measured link rate"},
                "sequential": {"ms_per_step": sum(seq_ms) / args.steps,
                               "value": n_tasks * args.steps / (sum(seq_ms) * 1e-3),
                               "note": "the three graphs one after another, no overlap between them"},
                "roofline": roof, "roofline_hbm": roof_hbm, "analysis_roofline": analysis_roof,
                "atomic_roofline": atomic_roof, "stencil_1d": stencil1d, "rects_1m": rects_1m,
                "spin_bodies": spin, "event_executor": events,
                "cpu_baseline": cpu, "clocks": clk,
                "gpu_launches": launches,
                "batched": batched, "served": served, "metg": metg, "async_nodes": async_nodes, "stitched": stitched,
                "wall_s_timed": wall,
                "phases_ms_per_graph": [{k: round(v, 4) for k, v in a.items()} for a in avg]}
        print(json.dumps(line), flush=True)
    for g in graphs:
        g.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--no-metg", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the SPIN-body and event-executor comparisons")
    ap.add_argument("--graph-steps", type=int, default=STEPS, help="profiling only: fewer steps per graph")
    ap.add_argument("--patterns", default=",".join(tg.PATTERNS), help="profiling only: subset of patterns")
    ap.add_argument("--case", default=None, choices=["served-batch"],
                    help="profiling only: run one named analysis case instead of the bench")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.case == "served-batch":
        return run_case_served_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
