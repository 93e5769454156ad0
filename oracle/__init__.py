"""CPU oracle for the dependence-analysis / actor-execution hot path.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product package.
"""
from .oracle import (  # noqa: F401
    BODY_CHECK,
    BODY_COUNTER,
    BODY_EMPTY,
    BODY_FMA,
    BODY_SPIN,
    alg1_run,
    analyze,
    analyze_intervals,
    build,
    csr_from_pairs,
    fma_bits,
    mix32,
    run_bodies,
    spin,
    topo_order,
)
