"""The shortcut of Sec. 6 (complete algorithm and complexity): a problem with
no state-only or terminal rows whose every stage's mixed rows leave no row on
x_i once u_i is projected out has X_i = R^n for all i, and its feasible-domain
scan is skipped.  The skipped path must give the scanned path's results bit for
bit and the oracle's within the parity tolerance; problems that fail the test
(a D_i row of zeros, terminal rows) must take the scan."""
import numpy as np
import pytest

import oracle
from paper_2407_05433_gb300 import eclqr, synth

pytestmark = pytest.mark.gpu
TOL = 1e-9
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


def problems():
    free = synth.config("mixed_only_n12", N=96)
    # same structure, but one stage has a mixed row with D = 0: that row binds x_i
    rng = np.random.default_rng(7)
    p = rng.integers(1, 4, size=64)
    zero_row = int(p[:10].sum())  # first row of stage 10
    bound = synth.make_problem(3, 64, 6, 3, p, np.zeros(65, dtype=np.int32), zero_D_rows=[zero_row])
    terminal = synth.config("single_n4", N=32)  # terminal rows: not eligible
    return [free, bound, terminal]


def run(pbs, scan_skip, chunk=8):
    b = eclqr.Batch(pbs, refine=2, chunk=chunk, scan_skip=scan_skip)
    try:
        b.run()
        return b.results(), b.scan_skipped()
    finally:
        b.close()


@pytest.mark.parametrize("chunk", [8, 5])
def test_skip_matches_scan_bit_for_bit_and_flags_the_right_problems(chunk):
    pbs = problems()
    r1, f1 = run(pbs, 1, chunk)
    r0, f0 = run(pbs, 0, chunk)
    assert f1.tolist() == [True, False, False]
    assert f0.tolist() == [False, False, False]
    for a, b in zip(r1, r0):
        assert a["status"] == b["status"] == 0
        for k in KEYS:
            assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k


def test_skipped_problem_matches_the_oracle():
    pbs = problems()
    res, flags = run(pbs, 1)
    assert flags[0]
    for pb, r in zip(pbs, res):
        s = oracle.solve(pb)
        assert s.ok
        for k in KEYS:
            e = rel(r[k], getattr(s, k))
            assert e <= TOL, f"{k}: rel err {e:.3e}"
        assert r["resid"] <= 1e-9


def test_full_size_skipped_instance_matches_the_oracle():
    """mixed_only_n12 at its full horizon (N=1024), the instance bench.py times the shortcut on."""
    pb = synth.config("mixed_only_n12")
    (r,), flags = run([pb], 1, chunk=0)
    assert flags[0]
    s = oracle.solve(pb)
    assert s.ok and r["status"] == 0
    for k in KEYS:
        e = rel(r[k], getattr(s, k))
        assert e <= TOL, f"{k}: rel err {e:.3e}"
    assert r["resid"] <= 1e-9
