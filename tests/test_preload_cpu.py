"""Every CUDA kernel of the library is loaded before a resident kernel starts.

With lazy module loading a kernel's first launch may wait for the device to go
idle, which a resident kernel (the serving kernel) never lets happen: a worker
launching a not-yet-loaded kernel would block for good. The server therefore
calls preload_all(), which calls each file's preload_* function. This test
reads the sources: every __global__ kernel of a file must be named in that
file's preload function (or in a helper it calls), and preload_all() must call
every preload function."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2508_16522_gb300", "csrc")

KERNEL = re.compile(r"__global__\s+void\s+(?:__launch_bounds__\([^)]*\)\s+)?(k_\w+)\s*\(")


def function_body(src, name):
    """The text between the braces of `name`'s definition (None if absent)."""
    m = re.search(r"\b" + re.escape(name) + r"\s*\([^)]*\)\s*(?:const\s*)?\{", src)
    if not m:
        return None
    depth, i = 1, m.end()
    while depth and i < len(src):
        depth += {"{": 1, "}": -1}.get(src[i], 0)
        i += 1
    return src[m.end():i - 1]


def sources():
    return {f: open(os.path.join(CSRC, f)).read() for f in sorted(os.listdir(CSRC)) if f.endswith(".cu")}


def test_every_kernel_is_preloaded():
    missing = []
    preloads = []
    for f, src in sources().items():
        kernels = sorted(set(KERNEL.findall(src)))
        if not kernels:
            continue
        names = [n for n in re.findall(r"^void (preload_\w+)\(\)", src, re.M) if n != "preload_all"]
        assert names, f"{f} defines kernels but no preload_* function"
        body = "".join(function_body(src, n) or "" for n in names)
        # one level of helpers called from the preload body (e.g. the list of
        # a kernel's template instantiations)
        for h in set(re.findall(r"\b(\w+)\(\)", body)):
            body += function_body(src, h) or ""
        preloads += names
        missing += [f"{f}: {k}" for k in kernels if not re.search(r"\b" + k + r"\b", body)]
    assert not missing, "kernels missing from their file's preload function: " + ", ".join(missing)
    prim = sources()["primitives.cu"]
    all_body = function_body(prim, "preload_all")
    assert all_body is not None
    assert not [p for p in preloads if p + "()" not in all_body], "preload_all() misses a preload function"


def test_server_preloads_everything_before_its_kernel():
    src = sources()["server.cu"]
    i_pre, i_launch = src.find("preload_all();"), src.find("launch_serve(p,")
    assert 0 <= i_pre < i_launch, "the server must call preload_all() before it launches the serving kernel"
