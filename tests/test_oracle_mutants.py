"""The oracle's pins must be able to fail: each plausible mistake below is
planted in a temporary copy of oracle.c (on the CPU), compiled, and must be
caught by the brute-force pairwise rule or a closed form."""
import os
import subprocess
import tempfile

import pytest

import oracle
from oracle import oracle as orc_mod
from paper_2508_16522_gb300 import tracegen as tg

from test_oracle_pins import as_set, brute_force_edges, tiny_traces

SRC = os.path.join(os.path.dirname(orc_mod.__file__), "oracle.c")

MUTANTS = {
    # joining a read/reduce run takes edges from the current run instead of the previous one
    "join_uses_last_run": ("for (int32_t k = 0; k < P->n; ++k)\n          if (vec64_push(&pairs, ((uint64_t)(uint32_t)P->m[k]",
                           "for (int32_t k = 0; k < L->n; ++k)\n          if (vec64_push(&pairs, ((uint64_t)(uint32_t)L->m[k]"),
    # read + reduce treated as read instead of write (O1)
    "combine_read_reduce": ("if (have == add && add != P_WRITE) return add;",
                            "if (have != P_WRITE && add != P_WRITE) return have;"),
    # consecutive writes merged into one run
    "writes_form_runs": ("if (L->n > 0 && L->kind == p && p != P_WRITE) {",
                         "if (L->n > 0 && L->kind == p) {"),
    # only the first member of a run gives edges to a newcomer
    "first_member_only": ("for (int32_t k = 0; k < L->n; ++k)\n          if (vec64_push(&pairs, ((uint64_t)(uint32_t)L->m[k]",
                          "for (int32_t k = 0; k < (L->n ? 1 : 0); ++k)\n          if (vec64_push(&pairs, ((uint64_t)(uint32_t)L->m[k]"),
    # explicit preds ignored
    "drop_explicit_preds": ("if (pred_off) {", "if (0) {"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "mut.c")
        so = os.path.join(d, "libmut.so")
        open(c, "w").write(src.replace(old, new))
        subprocess.check_call(["gcc", "-O1", "-std=c99", "-shared", "-fPIC", "-o", so, c, "-lm"])
        cases = tiny_traces() + [tg.stencil_1d(16, 6), tg.fig6_fixture()]
        wrong = 0
        for tr in cases:
            got = as_set(*oracle.analyze(tr, lib_path=so))
            if got != brute_force_edges(tr):
                wrong += 1
        assert wrong > 0, f"mutant {name} survived every pin"
