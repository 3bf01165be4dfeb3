"""The KKT residual (Sec. 9 definition), its refinement and non-finite data on the CUDA path, through
the C ABI, against the CPU oracle.

* eclqr_kkt_residual_parts against the oracle's residual, part by part (initial condition, dynamics,
  normalised equality rows, stationarity), at the solution and at points perturbed in one part.
* eclqr_refine on uneven-batch draws that need it: element by element against the oracle at 1e-9.
* A NaN in the data or in s_0: status NONFINITE and a NaN residual, on the GPU and in the oracle.
* The uneven-batch workload under the large-batch schedule (one chunk per problem): 512 distinct
  draws, every block against the oracle at 1e-9, every residual under its gate (1e-9, or for the
  draws listed in tests/golden/batched_uneven_floors.txt the floor of the problem itself).
"""
import os
from multiprocessing import get_context

import numpy as np
import pytest

import oracle
from paper_2407_05433_gb300 import eclqr, synth

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
KEYS = ("x", "u", "lam", "mu", "eta", "alpha")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2407_05433_gb300 import build as b
    b.build()
    eclqr.load()


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    if b.size == 0:
        return 0.0
    return float(np.max(np.abs(a - b)) / max(1.0, np.max(np.abs(b))))


def load_floors():
    """{index: gate} of the uneven-batch draws whose own FP64 floor exceeds the 1e-9 gate."""
    out = {}
    for ln in open(os.path.join(HERE, "golden", "batched_uneven_floors.txt")):
        if ln.startswith("#") or not ln.strip():
            continue
        j, N, n, rho, phi, ext = ln.split()
        out[int(j)] = max(1e-9, 4.0 * float(phi))
    return out


def _problem_with(pb, key, arr):
    q = pb.copy()
    setattr(q, key, arr)
    return q


def test_residual_parts_match_the_oracle_value_for_value():
    """At the solution both residuals are rounding noise below 1e-9 that agree to 1e-12 absolute.  Then
    one part at a time is
    made large -- s_0 passed to the residual (initial condition), c (dynamics), d (mixed rows,
    normalised), q (stationarity) -- and the four parts agree with the oracle's to 1e-12 relative."""
    import torch
    pbs = [synth.config("single_n4", N=30), synth.config("table1", N=20),
           synth.config("batched_uneven", index=5, N=40), synth.config("degenerate_n12", N=25)]
    b = eclqr.Batch(pbs)
    try:
        b.run()
        res = b.results()
        parts0 = b.residual_parts()
        for pb, r, p in zip(pbs, res, parts0):
            _, po = oracle.kkt_residual(pb, r["x"], r["u"], r["lam"], r["mu"], r["eta"], r["alpha"], parts=True)
            assert np.all(p <= 1e-9) and np.all(po <= 1e-9) and np.all(np.abs(p - po) <= 1e-12), (p, po)
        rng = np.random.default_rng(7)
        for key, part in (("s0", 0), ("c", 1), ("d", 2), ("qv", 3)):
            orig = b.d[key].clone()
            pert = orig + torch.from_numpy(rng.uniform(0.5, 1.5, orig.numel())).to(orig.device)
            if key == "s0":
                parts = b.residual_parts(s0=pert)
            else:
                b.d[key].copy_(pert)
                parts = b.residual_parts()
                b.d[key].copy_(orig)
            host = pert.cpu().numpy()
            off = 0
            for j, (pb, r) in enumerate(zip(pbs, res)):
                size = getattr(pb, key).size
                mod = _problem_with(pb, key, host[off:off + size].reshape(getattr(pb, key).shape))
                off += size
                _, po = oracle.kkt_residual(mod, r["x"], r["u"], r["lam"], r["mu"], r["eta"], r["alpha"],
                                            parts=True)
                if key == "d" and pb.d.size == 0:
                    continue
                assert po[part] > 1e-2, (key, po)
                for k in range(4):
                    assert abs(parts[j, k] - po[k]) <= 1e-12 * max(1.0, po[k]), (key, j, k, parts[j], po)
    finally:
        b.close()


# uneven-batch draws whose single pass leaves a residual far above 1e-9 (see the oracle pins)
REFINED_DRAWS = [252, 261, 612, 344, 616, 158]


def test_refinement_on_the_kkt_residual_matches_the_oracle():
    pbs = [synth.config("batched_uneven", index=j) for j in REFINED_DRAWS]
    b0 = eclqr.Batch(pbs, kkt_refine=0)
    try:
        b0.run()
        r0 = b0.results()
    finally:
        b0.close()
    assert max(r["resid"] for r in r0) > 1e-7   # a single pass misses the gate on these draws
    b = eclqr.Batch(pbs)
    try:
        b.run()
        res = b.results()
    finally:
        b.close()
    for pb, r in zip(pbs, res):
        s = oracle.solve(pb)
        assert s.ok and r["status"] == 0
        assert r["resid"] <= 1e-9
        for k in KEYS:
            assert rel(r[k], getattr(s, k)) <= 1e-9, k


def test_refinement_with_zero_passes_only_computes_the_residual():
    import torch
    pb = synth.config("batched_uneven", index=252)
    b = eclqr.Batch([pb], kkt_refine=0)
    try:
        b.build(); b.solve(); b.multipliers()
        torch.cuda.synchronize()
        before = {k: getattr(b, k).clone() for k in KEYS}
        b.refine()
        (after,) = b.results()
        for k in KEYS:
            assert np.array_equal(before[k].cpu().numpy()[:after[k].size], np.asarray(after[k]).ravel()), k
        b.residual()
        torch.cuda.synchronize()
        assert float(b.resid[0]) == after["resid"]
    finally:
        b.close()


def test_solve_after_refine_needs_a_new_build():
    """After a pass ran, the offset-dependent workspace is the last correction's: solve refuses until
    the next build.  Where no problem needed a pass, the workspace is untouched and solve runs."""
    b = eclqr.Batch([synth.config("batched_uneven", index=252)])
    try:
        b.run()
        with pytest.raises(RuntimeError, match="call out of order"):
            b.solve()
        b.build()
        b.solve()
    finally:
        b.close()
    b = eclqr.Batch([synth.config("single_n4", N=20)])
    try:
        b.run()
        assert float(b.resid[0]) <= 5e-10
        b.solve()
    finally:
        b.close()


@pytest.mark.parametrize("where", ["A", "d", "s0"])
def test_nonfinite_data_gives_status_and_nan_residual(where):
    """A NaN in one input: status NONFINITE and a NaN residual, on the GPU and in the oracle.  Every
    loop of the factorizations runs to bounds fixed by the dimensions, so NaN data only make NaN
    values; the check of the data in the build turns them into the status."""
    pbs = [synth.config("single_n4", N=16), synth.config("batched_uneven", index=3, N=12)]
    bad = pbs[0].copy()
    arr = getattr(bad, where).copy()
    arr.reshape(-1)[arr.size // 2] = np.nan
    setattr(bad, where, arr)
    b = eclqr.Batch([bad, pbs[1]])
    try:
        b.run()
        r = b.results()
    finally:
        b.close()
    assert eclqr.STATUS_NAMES[r[0]["status"]] == "nonfinite"
    assert np.isnan(r[0]["resid"])
    assert r[1]["status"] == 0 and r[1]["resid"] <= 1e-9     # the other problem of the batch is unaffected
    assert oracle.STATUS_NAMES[oracle.solve(bad).status] == "nonfinite"


def _oracle_job(j):
    import oracle as o
    from paper_2407_05433_gb300 import synth as sy
    pb = sy.config("batched_uneven", index=j)
    s = o.solve(pb)
    return j, s.status, {k: getattr(s, k) for k in KEYS}


def multiplier_gap(pb, r, sol):
    """|J'(y_gpu - y_oracle)|_inf: the stationarity rows of the multiplier difference alone (no costs, x =
    u = 0).  Small where the two multipliers differ only along a direction the KKT system leaves nearly
    free (a nearly rank-deficient constraint Jacobian)."""
    z = pb.copy()
    z.qv = np.zeros_like(pb.qv)
    z.rv = np.zeros_like(pb.rv)
    z.s0 = np.zeros_like(pb.s0)
    _, parts = oracle.kkt_residual(z, np.zeros_like(r["x"]), np.zeros_like(r["u"]), r["lam"] - sol["lam"],
                                   r["mu"] - sol["mu"], r["eta"] - sol["eta"], r["alpha"] - sol["alpha"],
                                   parts=True)
    return float(parts[3])


def test_uneven_batch_512_distinct_draws_default_schedule():
    """512 distinct draws (more than two problems per SM, so one chunk per problem, longest horizons
    first: the schedule of the full 4096-problem batch) against the oracle: x and u at 1e-9, every
    residual under 1e-9.  The multipliers match at 1e-9 too, or, where the constraint Jacobian is
    nearly rank-deficient and they are not fixed to that accuracy (the exact KKT solve itself differs
    from the refined oracle by 1e-9 on draw 129, at residuals of 2e-11), differ only by a vector w with
    |J'w| within twice the gate: equal modulo the near-null space of J', the comparison used for
    rank-deficient J.  A draw listed in tests/golden/batched_uneven_floors.txt has an FP64 floor of its
    own, 4 phi > 1e-9; there the bars are 4 phi (the refined oracle itself lies within phi of the exact
    KKT solution on every such draw but 250).  Draw 250's KKT matrix is too close to singular for its
    solution to be fixed to FP64 accuracy (two exact solves disagree in x at 1e-1); it is held to its
    status only."""
    floors = load_floors()
    idx = list(range(512))
    oracle.build_oracle()
    with get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        orc = {j: (st, sol) for j, st, sol in pool.map(_oracle_job, idx, chunksize=8)}
    pbs = [synth.config("batched_uneven", index=j) for j in idx]
    b = eclqr.Batch(pbs)
    try:
        b.run()
        res = b.results()
    finally:
        b.close()
    bad, modulo = [], []
    for j, r in zip(idx, res):
        st, sol = orc[j]
        assert st == 0 and r["status"] == 0, (j, st, r["status"])
        if j == 250:
            continue
        gate = floors.get(j, 1e-9)
        errs = {k: rel(r[k], sol[k]) for k in KEYS}
        primal_ok = errs["x"] <= gate and errs["u"] <= gate
        dual_ok = max(errs[k] for k in ("lam", "mu", "eta", "alpha")) <= gate
        if not dual_ok and multiplier_gap(pbs[j], r, sol) <= 2 * gate:
            dual_ok = True
            modulo.append(j)
        if r["resid"] > gate or not primal_ok or not dual_ok:
            bad.append((j, r["resid"], gate, errs))
    assert not bad, bad[:5]
    assert len(modulo) <= 8, modulo
