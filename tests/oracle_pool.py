"""Oracle work of the full-size tests spread over the host's cores.

The pool's processes are started with ``spawn`` (a process forked after CUDA
was initialised would hang), import only the oracle and the trace generator,
rebuild each graph from its seed, and return digests of the oracle's results,
so that little data crosses the process boundary."""
import hashlib
import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np

import oracle
from paper_2508_16522_gb300 import tracegen as tg


def digest(*arrays) -> str:
    h = hashlib.sha1()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def csr_digest(rp, col) -> str:
    return digest(np.asarray(rp, np.int64), np.asarray(col, np.int32))


def _batch_part(args):
    n_graphs, seed, idx, runs = args
    specs = tg.batch_graph_specs(n_graphs, seed=seed)
    out = []
    for k in idx:
        tr = tg.batch_graph(specs[k])
        s, d = oracle.analyze(tr)
        rp, col = oracle.csr_from_pairs(tr.n, s, d)
        st = o = None
        for _ in range(runs):
            st, o = oracle.run_bodies(tr, oracle.BODY_CHECK, state=st)
        out.append((k, csr_digest(rp, col), digest(st[:tr.n_cells].astype(np.int32), o[:tr.n].astype(np.int32))))
    return out


def batch_check_digests(n_graphs: int, seed: int, runs: int, procs: int = 0):
    """{graph: (CSR digest, CHECK state+outputs digest after `runs` sequential
    runs)} for every graph of tracegen.batch_graphs(n_graphs, seed=seed)."""
    procs = procs or os.cpu_count() or 1
    parts = [(n_graphs, seed, list(range(p, n_graphs, procs)), runs) for p in range(procs)]
    with ProcessPoolExecutor(max_workers=procs, mp_context=mp.get_context("spawn")) as ex:
        res = {}
        for part in ex.map(_batch_part, parts):
            for k, a, b in part:
                res[k] = (a, b)
    return res
