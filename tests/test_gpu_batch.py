"""Batched execution: many captured graphs in one persistent launch, each
replayed independently. Every graph's result in the batch must equal its
result alone (the oracle's sequential execution, repeated per replay)."""
import numpy as np
import pytest

import oracle
from paper_2508_16522_gb300 import grt
from paper_2508_16522_gb300 import tracegen as tg

from gpu_helpers import gpu_graph

pytestmark = pytest.mark.gpu


def _oracle_repeat(tr, body, reps, spin_iters=256, state_elems=None):
    st = np.zeros(state_elems, np.int32) if state_elems else None
    out = None
    for _ in range(reps):
        st, out = oracle.run_bodies(tr, body, state=st, spin_iters=spin_iters)
    return st, out


POLICIES = [grt.RT_EXEC_RING, grt.RT_EXEC_OWNED]


@pytest.mark.parametrize("policy", POLICIES)
@pytest.mark.parametrize("replays", [1, 3])
def test_mixed_batch_equals_each_graph_alone(replays, policy):
    traces, bodies = [], []
    for k in range(24):
        if k % 4 == 0:
            traces.append(tg.random_rects(grid=(30, 22), n=150 + 10 * k, rects=(1, 3), side=(1, 9), seed=100 + k))
            bodies.append(grt.RT_BODY_CHECK)
        elif k % 4 == 1:
            traces.append(tg.taskbench(32, 5 + k, tg.PATTERNS[k % 3], seed=k))
            bodies.append(grt.RT_BODY_SPIN)
        elif k % 4 == 2:
            traces.append(tg.stencil_1d(8, 3 + k, 64))
            bodies.append(grt.RT_BODY_COUNTER)
        else:
            traces.append(tg.taskbench(16, 9, "butterfly", encode="explicit"))
            bodies.append(grt.RT_BODY_EMPTY)
    graphs = []
    for tr, b in zip(traces, bodies):
        g = gpu_graph(tr, body=b, spin_iters=37, tile=(8, 8) if tr.ndim == 2 else (64, 1),
                      state_elems=8 if b == grt.RT_BODY_COUNTER else None)
        g.analyze()
        graphs.append(g)
    batch = grt.Batch(graphs)
    batch.exec_policy(policy)
    batch.execute(replays=replays)
    ms = batch.sync()
    assert ms > 0
    for tr, b, g in zip(traces, bodies, graphs):
        if b == grt.RT_BODY_CHECK:
            st, out = _oracle_repeat(tr, oracle.oracle.BODY_CHECK, replays)
            assert np.array_equal(g.state.cpu().numpy(), st), tr.name
            assert np.array_equal(g.out.cpu().numpy(), out), tr.name
        elif b == grt.RT_BODY_SPIN:
            want = np.array([oracle.spin(j, 37) for j in range(tr.n)], np.uint32).view(np.int32)
            assert np.array_equal(g.out.cpu().numpy(), want), tr.name
        elif b == grt.RT_BODY_COUNTER:
            st, _ = _oracle_repeat(tr, oracle.oracle.BODY_COUNTER, replays, state_elems=8)
            assert np.array_equal(g.state.cpu().numpy(), st), tr.name
    # the batch can run again (counters re-armed by the tasks themselves)
    batch.execute(replays=1)
    batch.sync()
    batch.close()
    for g in graphs:
        g.close()


@pytest.mark.parametrize("policy", POLICIES)
def test_batch_with_empty_and_single_task_graphs(policy):
    import torch
    empty = grt.Graph(2, [0, 0], [3, 3])
    empty.analyze()
    one = gpu_graph(tg._finish(2, [0, 0], [3, 3], [1], np.array([0, 0]), np.array([3, 3]),
                               np.array([1], np.uint8)), body=grt.RT_BODY_SPIN, spin_iters=5)
    one.analyze()
    big = gpu_graph(tg.taskbench(64, 30, "random"), body=grt.RT_BODY_SPIN, spin_iters=5)
    big.analyze()
    b = grt.Batch([empty, one, big])
    b.exec_policy(policy)
    b.execute(replays=4)
    b.sync()
    assert one.out.cpu().tolist() == [oracle.spin(0, 5)]
    want = np.array([oracle.spin(j, 5) for j in range(64 * 30)], np.uint32).view(np.int32)
    assert np.array_equal(big.out.cpu().numpy(), want)
    b.close()
    for g in (empty, one, big):
        g.close()
    del torch


@pytest.mark.parametrize("shape", [(0, 0, 0, 0, 0), (152, 2, 8, 8, 0), (304, 4, 32, 64, 0), (1, 1, 1, 0, 0),
                                   (0, 0, 0, 0, 1), (152, 8, 1, 0, 1), (7, 1, 4, 0, 1), (304, 8, 2, 0, 1),
                                   (1, 1, 1, 0, 1)])
def test_batch_launch_shapes_give_same_results(shape):
    """(blocks, warps, claim, keep, policy): the ring policy's shapes, and the
    owned policy's (claim = lanes per task), down to one block of one warp."""
    gs_tr = tg.batch_graphs(60, n_range=(64, 4096), seed=3)
    graphs = []
    for tr in gs_tr:
        g = gpu_graph(tr, body=grt.RT_BODY_SPIN, spin_iters=3, tile=(8, 8))
        g.analyze()
        graphs.append(g)
    b = grt.Batch(graphs)
    blocks, warps, claim, keep, policy = shape
    b.exec_policy(policy)
    b.execute(replays=2, blocks=blocks, warps=warps, claim=claim, keep=keep)
    b.sync()
    for tr, g in zip(gs_tr, graphs):
        want = np.array([oracle.spin(j, 3) for j in range(tr.n)], np.uint32).view(np.int32)
        assert np.array_equal(g.out.cpu().numpy(), want), tr.name
    b.close()
    for g in graphs:
        g.close()


def test_stacked_batch_equals_each_graph_alone():
    """Graphs stacked in bands of one domain are captured by ONE analysis; the
    batch made from it runs each graph and replays it independently. Each
    graph's part of the CSR equals its own oracle CSR, SPIN outputs count from
    the graph's own first task, and the CHECK state after 3 replays equals the
    oracle's 3 sequential runs of the whole stack (the graphs share no cell)."""
    from gpu_helpers import oracle_csr
    trs = [tg.random_rects(grid=(40, 30), n=200 + 30 * k, rects=(1, 3), side=(1, 9), seed=200 + k) for k in range(5)]
    trs += [tg.taskbench(32, 6 + k, tg.PATTERNS[k % 3], seed=k) for k in range(4)]
    st, off = tg.stack_bands(trs)
    for body, spin in ((grt.RT_BODY_SPIN, 21), (grt.RT_BODY_CHECK, 0)):
        g = gpu_graph(st, body=body, spin_iters=spin, tile=(8, 8))
        g.analyze()
        rp, col, ind = g.csr()
        for k, tr in enumerate(trs):
            a, b = int(off[k]), int(off[k + 1])
            rp_o, col_o, _ = oracle_csr(tr)
            mine = rp[a:b + 1].astype(np.int64) - int(rp[a])
            assert np.array_equal(mine, rp_o), tr.name
            assert np.array_equal(col[rp[a]:rp[b]] - a, col_o), tr.name
        batch = grt.Batch.stacked(g, off)
        batch.execute(replays=3)
        batch.sync()
        assert batch.counters()["tasks"] == 3 * st.n
        if body == grt.RT_BODY_SPIN:
            out = g.out.cpu().numpy()
            for k, tr in enumerate(trs):
                want = np.array([oracle.spin(j, spin) for j in range(tr.n)], np.uint32).view(np.int32)
                assert np.array_equal(out[off[k]:off[k + 1]], want), tr.name
        else:
            # each graph's part of the stack, with its own task ids, in the
            # stack's domain: the bodies see their own ids and the shared cells
            parts = []
            for k in range(len(trs)):
                a, b = int(off[k]), int(off[k + 1])
                r0, r1 = int(st.req_off[a]), int(st.req_off[b])
                parts.append(tg._finish(2, st.dom_lo, st.dom_hi, np.diff(st.req_off[a:b + 1]),
                                        st.lo[r0:r1].reshape(-1), st.hi[r0:r1].reshape(-1), st.priv[r0:r1]))
            s_o = np.zeros(st.n_cells, np.int32)
            outs = [None] * len(parts)
            for _ in range(3):
                for k, part in enumerate(parts):
                    s_o, outs[k] = oracle.run_bodies(part, oracle.oracle.BODY_CHECK, state=s_o)
            assert np.array_equal(g.state.cpu().numpy(), s_o)
            out = g.out.cpu().numpy()
            for k in range(len(parts)):
                assert np.array_equal(out[off[k]:off[k + 1]], outs[k][:trs[k].n]), trs[k].name
        batch.close()
        g.close()


def test_stacked_batch_refuses_graphs_that_share_cells():
    trs = [tg.random_rects(grid=(20, 20), n=60, rects=(1, 2), side=(2, 8), seed=300 + k) for k in range(2)]
    both = tg.concat(trs)  # same cells: edges join the two
    g = gpu_graph(both)
    g.analyze()
    with pytest.raises(grt.GrtError) as e:
        grt.Batch.stacked(g, [0, trs[0].n, both.n])
    assert e.value.status == grt.RT_ERR_INVALID
    g.close()


def test_capture_places_graphs_in_bands_itself():
    """rt_batch_capture: graphs given in their own domains (some offset), placed
    in bands by the library and analysed once. Each graph's part of the CSR
    equals its own oracle CSR; with the CHECK body the batch's state and
    outputs after 2 launches of 3 replays equal the oracle's 6 sequential runs
    of the same graphs placed on the host (each graph's tasks numbered from 0,
    as a batched body sees them); later launches come from the cached CUDA
    graph."""
    import torch
    traces = [tg.taskbench(32, 9, "random", seed=1), tg.random_rects(grid=(40, 17), n=300, side=(1, 12), seed=4),
              tg.taskbench(8, 30, "butterfly", seed=2), tg.random_rects(grid=(25, 31), n=200, side=(1, 9), seed=5)]
    # give the second graph an offset domain: the library must move it to its band
    t1 = traces[1]
    off = np.array([-7, 100], np.int64)
    traces[1] = tg._finish(2, t1.dom_lo + off, t1.dom_hi + off, np.diff(t1.req_off), (t1.lo + off).reshape(-1),
                           (t1.hi + off).reshape(-1), t1.priv, name="offset")
    host, _ = tg.stack_bands(traces)  # the same placement, on the host, for the oracle
    T = host.n
    state = torch.zeros(host.n_cells, dtype=torch.int32, device="cuda")
    out = torch.zeros(T, dtype=torch.int32, device="cuda")
    b = grt.Batch.capture(traces, body=grt.RT_BODY_CHECK, state=state, out=out, tile=(8, 8))
    rp, col, _ = b.graph_csr()
    toff = b.task_off
    for k, tr in enumerate(traces):
        a, z = int(toff[k]), int(toff[k + 1])
        s, d = oracle.analyze(tr)
        rp_o, col_o = oracle.csr_from_pairs(tr.n, s, d)
        assert np.array_equal(rp[a:z + 1].astype(np.int64) - int(rp[a]), rp_o), tr.name
        assert np.array_equal(col[rp[a]:rp[z]] - a, col_o), tr.name
    for _ in range(2):
        b.execute(replays=3)
        b.sync()
    assert b.info()["graph_launches"] >= 1
    # a batched body sees its graph's own task ids, in the stacked domain's cells
    st_o, out_o = _stacked_local_ids_state(traces, host, 6)
    assert np.array_equal(state.cpu().numpy(), st_o)
    assert np.array_equal(out.cpu().numpy(), out_o)
    # the owned policy (the batch as one DAG, a run barrier between replays)
    # continues from that state: 2 more launches of 2 replays
    b.exec_policy(grt.RT_EXEC_OWNED)
    for _ in range(2):
        b.execute(replays=2)
        b.sync()
    st_o, out_o = _stacked_local_ids_state(traces, host, 10)
    assert np.array_equal(state.cpu().numpy(), st_o)
    assert np.array_equal(out.cpu().numpy(), out_o)
    b.close()


def _stacked_local_ids_state(traces, host, runs):
    """The oracle's state and outputs for the stacked program when every task
    mixes in its id within its own graph (as a batched body does): the
    stacked program run graph by graph, each graph's launches relabelled from 0."""
    W = int(host.dom_hi[0]) + 1
    state = np.zeros(host.n_cells, np.int32)
    outs = []
    y = 0
    for tr in traces:
        h = int(tr.dom_hi[1] - tr.dom_lo[1]) + 1
        lo = tr.lo - tr.dom_lo + np.array([0, y])
        hi = tr.hi - tr.dom_lo + np.array([0, y])
        band = tg._finish(2, [0, 0], [W - 1, int(host.dom_hi[1])], np.diff(tr.req_off), lo.reshape(-1),
                          hi.reshape(-1), tr.priv)
        o = None
        for _ in range(runs):
            state, o = oracle.run_bodies(band, oracle.oracle.BODY_CHECK, state=state)
        outs.append(o[:tr.n])
        y += h
    return state, np.concatenate(outs)


def test_capture_one_dimensional_and_refusals():
    import torch
    traces = [tg.random_rects(grid=(300,), n=120, side=(1, 40), seed=s, ndim=1) for s in (1, 2, 3)]
    out = torch.zeros(sum(t.n for t in traces), dtype=torch.int32, device="cuda")
    b = grt.Batch.capture(traces, body=grt.RT_BODY_SPIN, spin_iters=9, out=out, tile=(64, 1))
    rp, col, _ = b.graph_csr()
    toff = b.task_off
    for k, tr in enumerate(traces):
        a, z = int(toff[k]), int(toff[k + 1])
        s, d = oracle.analyze(tr)
        rp_o, col_o = oracle.csr_from_pairs(tr.n, s, d)
        assert np.array_equal(rp[a:z + 1].astype(np.int64) - int(rp[a]), rp_o)
        assert np.array_equal(col[rp[a]:rp[z]] - a, col_o)
    b.execute(replays=2)
    b.sync()
    want = np.concatenate([np.array([oracle.spin(j, 9) for j in range(t.n)], np.uint32).view(np.int32)
                           for t in traces])
    assert np.array_equal(out.cpu().numpy(), want)
    b.close()
    # a rectangle outside its own graph's domain would reach the next band: refused
    bad = traces[0]
    hi = bad.hi.copy()
    hi[0, 0] = 305
    bad = tg._finish(1, bad.dom_lo, bad.dom_hi, np.diff(bad.req_off), bad.lo.reshape(-1), hi.reshape(-1), bad.priv)
    with pytest.raises(grt.GrtError) as e:
        grt.Batch.capture([bad, traces[1]], body=grt.RT_BODY_EMPTY)
    assert e.value.status == grt.RT_ERR_INVALID and "its own graph's domain" in str(e.value)
