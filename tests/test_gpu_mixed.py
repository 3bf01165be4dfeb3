"""Mixed precision (riccati_fp32 = 1): the square-root Riccati sweep in FP32, every other step in
FP64, refinement on the original KKT residual in FP64, and an FP64 redo of the problems the
refinement leaves above its tolerance.  The fixed point is the FP64 solution, so the bar is the
FP64 path's: every block against the oracle at 1e-9, the residual at 1e-9."""
import numpy as np
import pytest

import oracle
from paper_2407_05433_gb300 import eclqr, synth

pytestmark = pytest.mark.gpu
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


def run(pbs, **kw):
    b = eclqr.Batch(pbs, **kw)
    try:
        b.run()
        return b.results()
    finally:
        b.close()


def test_fp32_factors_are_in_use():
    """Without any refinement the FP32 factors leave errors far above the FP64 path's, so the mixed
    mode really runs its sweep in FP32."""
    pbs = [synth.config("diff_batch", index=j) for j in range(4)]
    r64 = run(pbs, refine=0, kkt_refine=0)
    r32 = run(pbs, refine=0, kkt_refine=0, riccati_fp32=1)
    e64 = max(rel(a["x"], b) for a, b in zip(r64, [oracle.solve(p).x for p in pbs]))
    e32 = max(rel(a["x"], b) for a, b in zip(r32, [oracle.solve(p).x for p in pbs]))
    assert e64 < 1e-10 and e32 > 1e-8, (e64, e32)


CASES = [
    ("single_n4", lambda: [synth.config("single_n4")]),
    ("diff_batch", lambda: [synth.config("diff_batch", index=j) for j in range(16)]),
    ("degenerate", lambda: [synth.config("degenerate_n12")]),
    ("long_shrunk", lambda: [synth.config("long_n16", N=2048)]),
    ("table1", lambda: [synth.config("table1", N=512)]),
    ("uneven", lambda: [synth.config("batched_uneven", index=j) for j in range(32)]),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_mixed_matches_the_oracle(name, make):
    pbs = make()
    res = run(pbs, riccati_fp32=1)
    for pb, r in zip(pbs, res):
        s = oracle.solve(pb)
        assert s.ok and r["status"] == 0
        assert r["resid"] <= 1e-9, r["resid"]
        for k in KEYS:
            assert rel(r[k], getattr(s, k)) <= 1e-9, (k, rel(r[k], getattr(s, k)))


def test_mixed_graph_replay_matches_eager():
    """The captured sequence (every pass and the FP64 redo recorded) gives the eager results to 1e-12."""
    import torch
    pbs = [synth.config("batched_uneven", index=j, N=40 + j) for j in range(6)]
    b = eclqr.Batch(pbs, riccati_fp32=1)
    try:
        b.run()
        torch.cuda.synchronize()
        ref = {k: getattr(b, k).clone() for k in KEYS}
        b.capture()
        for k in KEYS:
            getattr(b, k).zero_()
        b.replay()
        torch.cuda.synchronize()
        for k in KEYS:
            d = float((getattr(b, k) - ref[k]).abs().max()) / max(1.0, float(ref[k].abs().max()))
            assert d <= 1e-12, (k, d)
    finally:
        b.close()
