"""The stored algorithmic work of the benchmark workloads (tests/golden/workload_flops.json).

The file is written by tests/golden/make_workload_flops.py from the oracle alone; the bench
divides its entries by measured step times to report the useful FP64 rate.  These checks tie
the file to the oracle and to its own bookkeeping: the small workloads recount exactly, every
step total is the sum of the useful phases (0-6), and the uneven batch's one-pass entry differs
from the two-pass one only in phase 4 (rollout, refinement on the reduced residual, recovery)
and in phase 7 (the refinement on the KKT residual, which is not counted as useful work).
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2407_05433_gb300 import synth

PATH = os.path.join(os.path.dirname(__file__), "golden", "workload_flops.json")


@pytest.fixture(scope="module")
def stored():
    with open(PATH) as f:
        return json.load(f)["workloads"]


def test_step_totals_are_the_useful_phases(stored):
    for key, e in stored.items():
        ph = e["phase_flops"]
        assert len(ph) == 8, key
        assert e["step_flops"] == pytest.approx(sum(ph[:7]), rel=1e-12), key
        assert e["flops_per_stage"] == pytest.approx(e["step_flops"] / e["stages"], rel=1e-12), key
        assert all(v >= 0.0 for v in ph), key


@pytest.mark.parametrize("key,name,kw", [("single_n4", "single_n4", {}),
                                         ("table1_N1024", "table1", {"N": 1024})])
def test_small_workloads_recount_exactly(stored, key, name, kw):
    oracle.build_oracle()
    pb = synth.config(name, **kw)
    s = oracle.solve(pb)
    ph = [float(v) for v in s.phase_flops]
    e = stored[key]
    assert e["problems"] == 1 and e["stages"] == pb.N
    np.testing.assert_allclose(e["phase_flops"][:7], ph[:7], rtol=1e-12, atol=0.0)


def test_one_reduced_pass_changes_only_the_refinement_phases(stored):
    two, one = stored["batched_uneven"], stored["batched_uneven_refine1"]
    assert (one["problems"], one["stages"]) == (two["problems"], two["stages"])
    for k in (0, 1, 2, 3, 5, 6):
        assert one["phase_flops"][k] == pytest.approx(two["phase_flops"][k], rel=1e-12), k
    assert one["phase_flops"][4] < two["phase_flops"][4]
    assert one["step_flops"] < two["step_flops"]


def test_one_reduced_pass_recounts_on_a_draw():
    """Per draw, the one-pass count differs from the two-pass count in phase 4 alone, by one
    reduced refinement pass (a residual and a correction: positive work)."""
    oracle.build_oracle()
    pb = synth.config("batched_uneven", index=3)
    a = np.array(oracle.solve(pb, refine=2, kkt_refine=0).phase_flops, float)
    b = np.array(oracle.solve(pb, refine=1, kkt_refine=0).phase_flops, float)
    np.testing.assert_array_equal(np.delete(a, 4), np.delete(b, 4))
    assert b[4] < a[4]
