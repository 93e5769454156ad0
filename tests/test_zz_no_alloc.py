"""The allocation-free executor entry point (rt_execute_csr_static).

It serves callers that may not allocate device memory when they run a graph
(an arena that owns all device memory, a loop where cudaMalloc/cudaFree is not
allowed). Its output must equal the regular entry point's on the same graph,
on two calls in a row (the calls share one static scratch array, so the second
call checks that the first call's leftovers are re-initialised), and its
tickets must show every edge respected: the SPIN output depends on the task
alone, so the order check is what shows that the countdowns held."""
import numpy as np
import pytest

from paper_2508_16522_gb300 import grt
from paper_2508_16522_gb300 import tracegen as tg

from gpu_helpers import gpu_graph

pytestmark = pytest.mark.gpu


def _device_csr(g, torch):
    st = g.stats()
    n, e = st["n_tasks"], st["n_edges"]
    rp = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    col = torch.empty(max(e, 1), dtype=torch.int32, device="cuda")
    ind = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    grt._check(grt.load().rt_copy_csr(g.h, rp.data_ptr(), col.data_ptr(), ind.data_ptr()))
    return rp, col, ind, n, e


@pytest.mark.parametrize("make", [
    lambda: tg.taskbench(256, 200, "random", seed=4),
    lambda: tg.random_rects(grid=(96, 80), n=20000, rects=(1, 4), side=(1, 16), seed=12),
    lambda: tg.taskbench(1024, 256, "butterfly"),  # 262144 tasks: the maximum
])
def test_static_entry_matches_regular_entry(make):
    import torch
    tr = make()
    g = gpu_graph(tr, body=grt.RT_BODY_SPIN, spin_iters=64)
    g.analyze()
    g.execute()
    g.sync()
    ref = g.out.cpu().numpy().copy()
    rp, col, ind, n, e = _device_csr(g, torch)
    src = np.repeat(np.arange(n), np.diff(rp.cpu().numpy()))
    dst = col.cpu().numpy()[:e]
    for _ in range(2):
        out = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        tk = torch.full((2 * n,), -1, dtype=torch.int32, device="cuda")
        grt.rt_execute_csr_static(rp.data_ptr(), col.data_ptr(), ind.data_ptr(), n, e, 64, out.data_ptr(),
                                  tk.data_ptr())
        assert np.array_equal(out.cpu().numpy(), ref)
        t = tk.cpu().numpy().reshape(n, 2).astype(np.int64)
        assert np.array_equal(np.sort(t.reshape(-1)), np.arange(2 * n)), "a task did not run exactly once"
        assert np.all(t[src, 1] < t[dst, 0]), "an edge was not respected"
    # and without tickets
    out = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    grt.rt_execute_csr_static(rp.data_ptr(), col.data_ptr(), ind.data_ptr(), n, e, 64, out.data_ptr())
    assert np.array_equal(out.cpu().numpy(), ref)
    g.close()


def test_static_entry_rejects_oversize_and_malformed():
    import torch
    n = (1 << 18) + 1
    z = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(grt.GrtError) as e:
        grt.rt_execute_csr_static(z.data_ptr(), z.data_ptr(), z.data_ptr(), n, 0, 1, z.data_ptr())
    assert e.value.status == grt.RT_ERR_INVALID and "at most 262144" in str(e.value)
    # a backward column and a wrong in-degree are reported, not executed
    rp = torch.tensor([0, 1, 1], dtype=torch.int32, device="cuda")
    col = torch.tensor([0], dtype=torch.int32, device="cuda")
    ind = torch.tensor([1, 0], dtype=torch.int32, device="cuda")
    out = torch.zeros(2, dtype=torch.int32, device="cuda")
    with pytest.raises(grt.GrtError) as e:
        grt.rt_execute_csr_static(rp.data_ptr(), col.data_ptr(), ind.data_ptr(), 2, 1, 1, out.data_ptr())
    assert "later task" in str(e.value)
    col = torch.tensor([1], dtype=torch.int32, device="cuda")
    ind = torch.tensor([0, 0], dtype=torch.int32, device="cuda")
    with pytest.raises(grt.GrtError) as e:
        grt.rt_execute_csr_static(rp.data_ptr(), col.data_ptr(), ind.data_ptr(), 2, 1, 1, out.data_ptr())
    assert "indeg" in str(e.value)
    bad_rp = torch.tensor([0, 5, 1], dtype=torch.int32, device="cuda")
    with pytest.raises(grt.GrtError) as e:
        grt.rt_execute_csr_static(bad_rp.data_ptr(), col.data_ptr(), ind.data_ptr(), 2, 1, 1, out.data_ptr())
    assert "row_ptr" in str(e.value)
