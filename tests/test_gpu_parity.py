"""GPU parity: libgrt (through the C ABI) against the CPU oracle.

Edge sets are compared as canonical CSR arrays (bit-exact: all of this is
integer work) and bodies by final state and per-task outputs, which must equal
sequential program-order execution.
"""
import numpy as np
import pytest

import oracle
from paper_2508_16522_gb300 import grt
from paper_2508_16522_gb300 import tracegen as tg

from gpu_helpers import assert_csr_equal, gpu_graph, oracle_csr, random_traces_small

pytestmark = pytest.mark.gpu


def test_fig6c_fixture():
    tr = tg.fig6_fixture()
    g = gpu_graph(tr, tile=(1, 1))
    g.analyze()
    rp, col, ind = assert_csr_equal(g, tr)
    assert ind.tolist() == [0, 1, 1, 2]
    g.execute()
    g.sync()
    g.close()


@pytest.mark.parametrize("tile", [(1024, 1), (256, 1), (100, 1), (17, 1)])
def test_stencil_1d_counter(tile):
    tr = tg.stencil_1d()
    g = gpu_graph(tr, body=grt.RT_BODY_COUNTER, tile=tile, state_elems=16)
    g.analyze()
    assert_csr_equal(g, tr)
    assert g.stats()["n_edges"] == 2985
    g.execute()
    g.sync()
    assert g.state.cpu().tolist() == [100] * 16
    g.replay(3)
    g.sync()
    assert g.state.cpu().tolist() == [400] * 16
    g.close()


@pytest.mark.parametrize("pattern", tg.PATTERNS)
@pytest.mark.parametrize("encode", ["region", "explicit"])
@pytest.mark.parametrize("tile", [(16, 16), (5, 7), (64, 4), (1, 1)])
def test_taskbench_small(pattern, encode, tile):
    tr = tg.taskbench(64, 40, pattern, seed=11, encode=encode)
    g = gpu_graph(tr, tile=tile)
    g.analyze()
    assert_csr_equal(g, tr)
    g.close()


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 4), (3, 5)])
def test_random_traces_csr_and_check_body(tile):
    for tr in random_traces_small(12):
        t = tile if tr.ndim == 2 else (tile[0] * tile[1], 1)
        g = gpu_graph(tr, body=grt.RT_BODY_CHECK, tile=t)
        g.analyze()
        assert_csr_equal(g, tr)
        g.execute()
        g.sync()
        st, out = oracle.run_bodies(tr, oracle.oracle.BODY_CHECK)
        assert np.array_equal(g.state.cpu().numpy(), st[:tr.n_cells]), tr.name
        assert np.array_equal(g.out.cpu().numpy(), out[:tr.n]), tr.name
        g.close()


def test_tiny_exhaustive_privilege_mixes():
    from test_oracle_pins import tiny_traces
    for tr in tiny_traces():
        for tile in ((1, 1), (4, 4)) if tr.ndim == 2 else ((1, 1), (5, 1)):
            g = gpu_graph(tr, tile=tile)
            g.analyze()
            assert_csr_equal(g, tr)
            g.close()


def test_long_runs_and_many_predecessors():
    """A cell read by 200 tasks then written (>= 3-member runs, >64 preds of one
    task: hash-list overflow), and one task with 70 rectangles in one tile
    (group longer than the 32-entry stage)."""
    n_read = 200
    lo = [[5, 5]] * n_read + [[0, 0]] + [[k % 8, k // 8] for k in range(70)] + [[5, 5]]
    hi = [[5, 5]] * n_read + [[15, 15]] + [[k % 8, k // 8] for k in range(70)] + [[6, 6]]
    priv = [0] * n_read + [1] + [k % 3 for k in range(70)] + [2]
    counts = [1] * n_read + [1, 70, 1]
    tr = tg._finish(2, [0, 0], [15, 15], counts, np.array(lo).reshape(-1), np.array(hi).reshape(-1),
                    np.array(priv, np.uint8), name="longruns")
    for tile in ((16, 16), (4, 4), (2, 3)):
        g = gpu_graph(tr, body=grt.RT_BODY_CHECK, tile=tile)
        g.analyze()
        assert_csr_equal(g, tr)
        g.execute()
        g.sync()
        st, out = oracle.run_bodies(tr, oracle.oracle.BODY_CHECK)
        assert np.array_equal(g.state.cpu().numpy(), st) and np.array_equal(g.out.cpu().numpy(), out)
        g.close()


def test_pair_buffer_overflow_reruns_once():
    """A run of K readers then a run of K reducers over the same 4 tiles: every
    reducer follows every reader, so each tile yields K^2 candidate pairs from
    only 2K entries, far more than the first guess for the pair buffer. The
    sweep overflows, reports what it reserved, and the rerun must fit and give
    the oracle's CSR. Overlapping smaller boxes on top stress chunk splits."""
    K = 256
    rng = np.random.default_rng(7)
    lo = [[0, 0]] * (2 * K)
    hi = [[31, 31]] * (2 * K)
    priv = [0] * K + [2] * K
    for k in range(300):  # then many small overlapping boxes of mixed kinds
        x, y = rng.integers(0, 30, 2)
        lo.append([x, y])
        hi.append([x + rng.integers(0, 3), y + rng.integers(0, 3)])
        priv.append(int(rng.integers(0, 3)))
    counts = [1] * len(priv)
    tr = tg._finish(2, [0, 0], [31, 31], counts, np.array(lo).reshape(-1), np.array(hi).reshape(-1),
                    np.array(priv, np.uint8), name="pair_overflow")
    ref = oracle_csr(tr)
    for tile in ((16, 16), (8, 8)):
        g = gpu_graph(tr, tile=tile)
        g.analyze()
        assert_csr_equal(g, tr, ref)
        st = g.stats()
        assert st["n_pairs"] > 4 * st["n_entries"], st  # the first guess (2 x entries, >= 64K) was exceeded
        g.close()


def _dense_overflow_trace(K):
    """K readers then K reducers over the whole 64 x 64 domain, then small mixed
    boxes: at 8 x 8 tiles every task covers 64 tiles (64 binned entries per
    task: the pair-key filter is on), and each tile finds the same K^2 pairs."""
    rng = np.random.default_rng(11)
    lo = [[0, 0]] * (2 * K)
    hi = [[63, 63]] * (2 * K)
    priv = [0] * K + [2] * K
    for k in range(200):
        x, y = rng.integers(0, 62, 2)
        lo.append([x, y])
        hi.append([x + rng.integers(0, 2), y + rng.integers(0, 2)])
        priv.append(int(rng.integers(0, 3)))
    return tg._finish(2, [0, 0], [63, 63], [1] * len(priv), np.array(lo).reshape(-1), np.array(hi).reshape(-1),
                      np.array(priv, np.uint8), name=f"dense_{K}")


@pytest.mark.parametrize("K", [64, 512])
def test_pair_filter_on_dense_inputs(K):
    """Dense inputs go through the pair-key filter: the CSR is the oracle's. At
    K = 64 far fewer pairs are written than the tiles find. At K = 512 (a
    reducer with 512 predecessors in every tile: past the per-task list, so
    they are written unfiltered) the pairs overflow the first guess for the
    buffer, the flagged tiles are swept again without the filter (a pair whose
    first write fell past the buffer's end is already in the table), and
    nothing is lost."""
    tr = _dense_overflow_trace(K)
    ref = oracle_csr(tr)
    g = gpu_graph(tr, tile=(8, 8))
    g.analyze()
    assert_csr_equal(g, tr, ref)
    st = g.stats()
    assert st["pair_filter_bits"] >= 16, st
    assert st["n_entries"] >= 16 * tr.n, st
    found = K * K * 64  # the readers-to-reducers pairs every one of the 64 tiles finds
    if K == 64:  # fewer distinct pairs than table slots: nearly every repeat is dropped
        assert st["n_pairs"] < found // 4, st
    else:  # past the first guess: the rerun ran
        assert st["n_pairs"] > 2 * st["n_entries"], st
    g.close()
    # the same launches sparse enough for no filter give the same CSR
    g = gpu_graph(tr, tile=(64, 64))
    g.analyze()
    assert_csr_equal(g, tr, ref)
    assert g.stats()["pair_filter_bits"] == 0
    g.close()


@pytest.mark.parametrize("tile", [(16, 16), (32, 32), (16, 8)])
def test_dense_tiles_with_several_rectangles_per_task(tile):
    """Dense tiles (swept as segments, one lane per class row) whose tasks hold
    up to 4 rectangles that often overlap one another in the same rows (one
    combined privilege per cell), with runs that reach back over many staged
    windows: the CSR and the CHECK body's results are the oracle's."""
    for seed, side in ((21, (4, 40)), (22, (8, 64))):
        tr = tg.random_rects(grid=(64, 48), n=700, rects=(1, 4), side=side, seed=seed)
        g = gpu_graph(tr, body=grt.RT_BODY_CHECK, tile=tile)
        g.analyze()
        assert_csr_equal(g, tr)
        g.execute()
        g.sync()
        st, out = oracle.run_bodies(tr, oracle.oracle.BODY_CHECK)
        assert np.array_equal(g.state.cpu().numpy(), st[:tr.n_cells]), tr.name
        assert np.array_equal(g.out.cpu().numpy(), out[:tr.n]), tr.name
        g.close()


def _max_classes(tr, tile):
    """Largest class grid (column classes x row classes) of any tile: the
    boundaries of the rectangles falling inside each tile, counted on the host."""
    tw, th = tile
    cuts = {}
    for (x0, y0), (x1, y1) in zip(tr.lo, tr.hi):
        for ty in range(y0 // th, y1 // th + 1):
            for tx in range(x0 // tw, x1 // tw + 1):
                cx, cy = cuts.setdefault((tx, ty), (set(), set()))
                for v, base, side, st in ((x0, tx * tw, tw, cx), (x1 + 1, tx * tw, tw, cx),
                                          (y0, ty * th, th, cy), (y1 + 1, ty * th, th, cy)):
                    if base < v < base + side:
                        st.add(v)
    return max((len(a) + 1) * (len(b) + 1) for a, b in cuts.values())


def test_large_tiles_sweep_class_grids_in_strips():
    """Tiles up to 128x128: small rectangles make class grids larger than the
    1024 cells a warp keeps, so those tiles are swept in strips of class rows."""
    tr = tg.random_rects(grid=(200, 150), n=1500, rects=(1, 3), side=(1, 6), seed=21)
    ref = oracle_csr(tr)
    for tile in ((64, 64), (128, 32), (128, 128), (32, 128)):
        assert _max_classes(tr, tile) > 1024, tile
        g = gpu_graph(tr, body=grt.RT_BODY_CHECK, tile=tile)
        g.analyze()
        assert_csr_equal(g, tr, ref)
        g.execute()
        g.sync()
        st, out = oracle.run_bodies(tr, oracle.oracle.BODY_CHECK)
        assert np.array_equal(g.state.cpu().numpy(), st) and np.array_equal(g.out.cpu().numpy(), out)
        g.close()


def test_big_rectangles_on_large_tiles():
    """Rectangles with sides log-uniform 16..512 on a 512^2 grid (the shape of
    the 1M-launch 4096^2 workload, scaled down): most tiles have few classes,
    so whole-tile rectangles cost one class each."""
    tr = tg.random_rects(grid=(512, 512), n=500, rects=(1, 4), side=(16, 512), seed=22)
    ref = oracle_csr(tr)
    for tile in ((16, 16), (64, 64), (128, 128)):
        g = gpu_graph(tr, tile=tile)
        g.analyze()
        assert_csr_equal(g, tr, ref)
        g.close()


def test_edge_cases():
    import torch
    # empty graph
    g = grt.Graph(2, [0, 0], [9, 9])
    g.analyze()
    g.execute()
    g.sync()
    rp, col, ind = g.csr()
    assert rp.tolist() == [0] and len(col) == 0
    g.close()
    # tasks without rectangles (all roots), one rect covering the domain
    tr = tg._finish(2, [-3, 7], [20, 40], [0, 0, 1, 0, 1],
                    np.array([-3, 7, -3, 7]), np.array([20, 40, 0, 10]), np.array([1, 0], np.uint8))
    for tile in ((16, 16), (128, 8)):
        g = gpu_graph(tr, body=grt.RT_BODY_CHECK, tile=tile)
        g.analyze()
        assert_csr_equal(g, tr)
        g.execute()
        g.sync()
        g.close()
    # several appended batches, mixing explicit preds and regions, host and device
    parts = [tg.taskbench(32, 6, "stencil", encode="region"), tg.taskbench(32, 6, "random", encode="explicit"),
             tg.taskbench(32, 6, "butterfly", encode="region")]
    whole = tg.concat(parts)
    g = grt.Graph(2, whole.dom_lo, whole.dom_hi, tile=(8, 8))
    base = 0
    for k, p in enumerate(parts):
        if p.pred is not None:
            p = tg._finish(2, p.dom_lo, p.dom_hi, np.diff(p.req_off), p.lo.reshape(-1), p.hi.reshape(-1), p.priv,
                           pred_counts=np.diff(p.pred_off), pred=p.pred + base)
        g.launch_trace(p, device=(k == 1))
        base += p.n
    g.analyze()
    assert_csr_equal(g, whole)
    g.close()
    del torch


def test_device_validation_reports_invalid():
    import torch
    tr = tg.taskbench(16, 4, "stencil")
    bad_hi = tr.hi.copy()
    bad_hi[3, 0] = 99  # outside the 16-wide domain
    g = grt.Graph(2, tr.dom_lo, tr.dom_hi)
    g.launch(torch.from_numpy(tr.req_off).cuda(), torch.from_numpy(tr.lo).cuda(), torch.from_numpy(bad_hi).cuda(),
             torch.from_numpy(tr.priv).cuda())
    with pytest.raises(grt.GrtError) as e:
        g.analyze()
    assert e.value.status == grt.RT_ERR_INVALID and "outside" in str(e.value)
    g.close()
    # deferred host validation of a backward-pointing pred
    g = grt.Graph(2, [0, 0], [1, 1])
    g.launch(np.zeros(3, np.int32), np.zeros((0, 2), np.int64), np.zeros((0, 2), np.int64), np.zeros(0, np.uint8),
             np.array([0, 0, 1], np.int32), np.array([1], np.int32), defer_check=True)
    with pytest.raises(grt.GrtError) as e:
        g.analyze()
    assert "predecessor" in str(e.value)
    g.close()


def test_spin_and_empty_bodies():
    tr = tg.taskbench(128, 30, "butterfly")
    g = gpu_graph(tr, body=grt.RT_BODY_SPIN, spin_iters=256)
    g.analyze()
    g.execute()
    g.sync()
    want = np.array([oracle.spin(j, 256) for j in range(tr.n)], np.uint32).view(np.int32)
    assert np.array_equal(g.out.cpu().numpy(), want)
    g.close()


def test_tickets_respect_every_edge():
    for tr in [tg.taskbench(256, 60, "random"), tg.random_rects(grid=(64, 64), n=3000, side=(2, 24), seed=5)]:
        g = gpu_graph(tr, flags=grt.RT_GRAPH_TICKETS)
        g.analyze()
        g.execute()
        g.sync()
        t = g.tickets()
        rp, col, _ = g.csr()
        src = np.repeat(np.arange(tr.n), np.diff(rp))
        assert (t[:, 0] < t[:, 1]).all()
        assert (t[src, 1] < t[col, 0]).all(), "a task started before one of its predecessors finished"
        assert sorted(np.concatenate([t[:, 0], t[:, 1]]).tolist()) == list(range(2 * tr.n))
        g.close()


def test_replay_equals_sequential_repeats():
    tr = tg.random_rects(grid=(40, 30), n=500, rects=(1, 3), side=(1, 12), seed=9)
    g = gpu_graph(tr, body=grt.RT_BODY_CHECK, tile=(8, 8))
    g.analyze()
    g.replay(3)
    g.sync()
    st = None
    for _ in range(3):
        st, out = oracle.run_bodies(tr, oracle.oracle.BODY_CHECK, state=st)
    assert np.array_equal(g.state.cpu().numpy(), st) and np.array_equal(g.out.cpu().numpy(), out)
    # and again through the cached CUDA graph
    g.replay(3)
    g.sync()
    for _ in range(3):
        st, out = oracle.run_bodies(tr, oracle.oracle.BODY_CHECK, state=st)
    assert np.array_equal(g.state.cpu().numpy(), st)
    g.close()


def test_bounded_wait_timeout_and_recovery():
    tr = tg.taskbench(64, 20, "stencil")
    g = gpu_graph(tr, body=grt.RT_BODY_SPIN, spin_iters=4, timeout_ns=300_000_000)
    g.analyze()
    g.hold_task(64 * 10 + 5)  # never becomes ready
    g.execute()
    with pytest.raises(grt.GrtError) as e:
        g.sync()
    assert e.value.status == grt.RT_ERR_TIMEOUT
    # the context is still usable and the next run re-initialises the counters
    g.execute()
    g.sync()
    want = np.array([oracle.spin(j, 4) for j in range(tr.n)], np.uint32).view(np.int32)
    assert np.array_equal(g.out.cpu().numpy(), want)
    g.close()


@pytest.mark.parametrize("pattern", tg.PATTERNS)
def test_taskbench_full_size(pattern):
    """width 1024 x 1000 steps, region encoding, the benchmark's launch
    configuration: CSR bit-exact against the oracle."""
    tr = tg.taskbench(1024, 1000, pattern)
    g = gpu_graph(tr, flags=grt.RT_GRAPH_TICKETS)
    g.analyze()
    rp, col, ind = assert_csr_equal(g, tr)
    want = {"stencil": 3_066_930, "butterfly": 2_045_952, "random": 5_114_880}[pattern]
    assert len(col) == want
    g.execute()
    g.sync()
    t = g.tickets()
    src = np.repeat(np.arange(tr.n), np.diff(rp))
    assert (t[src, 1] < t[col, 0]).all()
    g.close()


def test_microbench_reports_plausible_rooflines():
    from gpu_helpers import ensure_built
    ensure_built()
    mb = grt.rt_microbench_atomics()
    assert 50 < mb["dep_atomic_ns"] < 20000
    assert 50 < mb["dep_l2_load_ns"] < 20000
    for k in ("scatter_atomic_gops", "scatter_red_gops", "contended_atomic_gops", "contended_warp_agg_gops"):
        assert 0.01 < mb[k] < 10000, (k, mb[k])


def test_concurrent_analyses_with_different_tiles():
    """Graphs analysed at the same time from several host threads, each on its
    own stream with its own tile (so its own shared-memory need), give the
    oracle's CSR: per-kernel launch limits set by one thread must not fail
    another's launch."""
    import threading
    import torch
    trs = [tg.random_rects(grid=(256, 192), n=3000, rects=(1, 4), side=(1, 40), seed=s) for s in range(4)]
    refs = [oracle_csr(t) for t in trs]
    tiles = [(8, 8), (32, 32), (16, 16), (64, 16)]
    streams = [torch.cuda.Stream() for _ in trs]
    graphs = [gpu_graph(t, tile=tl, stream=st) for t, tl, st in zip(trs, tiles, streams)]
    errors = []

    def work(i):
        try:
            for _ in range(5):
                graphs[i].clear()
                graphs[i].launch_trace(trs[i])
                graphs[i].analyze()
        except Exception as e:  # surfaced below
            errors.append(repr(e))

    th = [threading.Thread(target=work, args=(i,)) for i in range(len(trs))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors, errors
    for g, t, ref in zip(graphs, trs, refs):
        assert_csr_equal(g, t, ref)
        g.close()


@pytest.mark.parametrize("readers", [5, 300, 1024, 1500])
def test_csr_by_buckets_and_by_pair_sort(readers):
    """A write of one cell followed by `readers` reads of it: the writer's row
    holds `readers` candidate pairs. Rows of at most 32 pairs are sorted by one
    thread, up to 1024 by a warp in shared memory, longer ones send the whole
    graph to the radix sort of all pairs; every path gives the oracle's CSR,
    with a Task Bench graph (short rows) on the bucket path too."""
    n = readers + 2
    lo = np.zeros(n, np.int64)
    lo[-1] = 1  # an unrelated task on another cell
    pv = np.array([1] + [0] * readers + [1], np.uint8)
    tr = tg._finish(1, [0], [7], np.ones(n), lo, lo, pv, name=f"fanout{readers}")
    g = gpu_graph(tr, tile=(8, 1))
    g.analyze()
    assert_csr_equal(g, tr)
    assert g.stats()["csr_by_buckets"] == (1 if readers <= 1024 else 0)
    g.close()
    tb = tg.taskbench(128, 40, "random", seed=readers)
    g = gpu_graph(tb)
    g.analyze()
    assert_csr_equal(g, tb)
    assert g.stats()["csr_by_buckets"] == 1
    g.close()
