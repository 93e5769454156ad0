"""Builds libgrt.so (the CUDA kernels + C ABI) for sm_103a, in-tree.

Each translation unit under csrc/ is compiled by nvcc in parallel, then linked
into paper_2508_16522_gb300/_lib/libgrt.so. Nothing is cached across machines:
the GPU machine (aarch64) and this container (x86_64) each build their own copy.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(HERE, "_lib")
SO = os.path.join(LIBDIR, "libgrt.so")
SOURCES = ["primitives.cu", "analysis.cu", "sweep.cu", "exec.cu", "static_exec.cu", "microbench.cu", "serve.cu", "server.cu", "tune.cu", "events.cu", "kernels.cu", "stitch.cu", "api.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(verbose: bool):
    f = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC] + ARCH
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    deps = [src, os.path.join(INCLUDE, "grt.h")] + [os.path.join(CSRC, h) for h in os.listdir(CSRC)
                                                      if h.endswith(".cuh")]
    return any(os.path.getmtime(d) > os.path.getmtime(obj) for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(LIBDIR, exist_ok=True)
    cc = nvcc()
    objs, jobs = [], []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(LIBDIR, s.replace(".cu", ".o"))
        objs.append(obj)
        if force or verbose or _stale(obj, src):
            jobs.append([cc, "-c", src, "-o", obj] + _flags(verbose))
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        for cmd, r in zip(jobs, results):
            if verbose or r.returncode:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode:
                raise RuntimeError("nvcc failed: " + " ".join(cmd))
    if force or jobs or not os.path.exists(SO):
        tmp = SO + f".tmp{os.getpid()}"
        subprocess.check_call([cc, "-shared", "-o", tmp] + objs + ARCH + ["-lcudart", "-Xcompiler", "-pthread"])
        os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
