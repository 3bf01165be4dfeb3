"""Can the reduced LQR's factors be formed in FP32 and the result refined in FP64?

A CPU study on the oracle's reduced problems (Sec. 5.3 data: Abar, Bbar,
cbar, Qbar, Mbar, Rbar, qbar, rbar), for the mixed-precision form in which the
square-root Riccati factors are computed in FP32 and classical iterative
refinement on the reduced KKT residual runs in FP64 with those factors.

The factors come from the square-root recursion: with G'G the stage Hessian
[[Rbar, Mbar'], [Mbar, Qbar]] (order v, z) and P_{i+1} = R_{i+1}'R_{i+1}, the
Householder QR of [G ; R_{i+1}Bbar | R_{i+1}Abar] gives R_vv, R_vz and R_i,
hence K_i = -R_vv^{-1}R_vz and H_uu = R_vv'R_vv.  Each solve with them is the
textbook two-pass LQR solve for given offsets (closed-loop p recursion,
forward rollout, costate lambda_i = P_i z_i + p_i); each refinement pass
evaluates the stage-wise KKT residual (stationarity in z and v, dynamics) in
FP64 and solves for the correction with the same factors.

The finding these tests pin: refinement converges from FP32 factors on the
well-conditioned differentiable-batch draw (n = 16, four mixed rows), but on
the degenerate n = 12 instance and on uneven-batch draws the reduced problem
is too ill-conditioned for FP32 factors (the first pass with FP64 factors
contracts the error there by only 1.6e-9, an effective condition near 1e7),
so the iteration does not reach the 1e-9 tolerance.  The CUDA path therefore
computes every factor in FP64.
"""
import numpy as np
import pytest

import oracle
from paper_2407_05433_gb300 import synth


def _reduced(pb):
    sol = oracle.solve(pb, debug=True, refine=4)
    assert sol.ok
    d = sol.debug
    nb, mb, N = d["nbar"], d["mbar"], pb.N
    blk = dict(
        A=[d["Abar"][i][:nb[i + 1], :nb[i]] for i in range(N)],
        B=[d["Bbar"][i][:nb[i + 1], :mb[i]] for i in range(N)],
        c=[d["cbar"][i][:nb[i + 1]] for i in range(N)],
        Q=[d["Qbar"][i][:nb[i], :nb[i]] for i in range(N + 1)],
        M=[d["Mbar"][i][:nb[i], :mb[i]] for i in range(N)],
        R=[d["Rbar"][i][:mb[i], :mb[i]] for i in range(N)],
        q=[d["qbar"][i][:nb[i]] for i in range(N + 1)],
        r=[d["rbar"][i][:mb[i]] for i in range(N)],
        z=[d["z"][i][:nb[i]] for i in range(N + 1)],
        v=[d["v"][i][:mb[i]] for i in range(N)])
    return blk, N


def _sqrt_riccati(b, N, dt):
    """Square-root Riccati factors computed in precision dt, returned in FP64."""
    P, K, U = [None] * (N + 1), [None] * N, [None] * N
    nN = b["Q"][N].shape[0]
    Rn = np.linalg.cholesky(b["Q"][N]).T.astype(dt) if nN else np.zeros((0, 0), dt)
    P[N] = (Rn.T @ Rn).astype(np.float64)
    for i in range(N - 1, -1, -1):
        A, B, Q, M, R = b["A"][i], b["B"][i], b["Q"][i], b["M"][i], b["R"][i]
        a, mm = A.shape[1], B.shape[1]
        G = np.linalg.cholesky(np.block([[R, M.T], [M, Q]])).T.astype(dt)
        S = np.vstack([G, np.hstack([Rn @ B.astype(dt), Rn @ A.astype(dt)])]).astype(dt)
        F = np.linalg.qr(S, mode="r").astype(dt)
        Rvv, Rvz, Rn = F[:mm, :mm], F[:mm, mm:mm + a], F[mm:mm + a, mm:mm + a]
        if Rn.shape[0] < a:
            Rn = np.vstack([Rn, np.zeros((a - Rn.shape[0], a), dt)])
        K[i] = (-np.linalg.solve(Rvv, Rvz)).astype(np.float64) if mm else np.zeros((0, a))
        U[i] = Rvv.astype(np.float64)
        P[i] = (Rn.T @ Rn).astype(np.float64)
    return P, K, U


def _solve(b, N, fac, q, r, c, z0):
    """LQR solve for offsets (q, r, c) with fixed factors, in FP64."""
    P, K, U = fac
    p, kf = [None] * (N + 1), [None] * N
    p[N] = q[N]
    for i in range(N - 1, -1, -1):
        A, B = b["A"][i], b["B"][i]
        w = P[i + 1] @ c[i] + p[i + 1]
        if B.shape[1]:
            h = r[i] + B.T @ w
            kf[i] = -np.linalg.solve(U[i], np.linalg.solve(U[i].T, h))
            p[i] = q[i] + (A + B @ K[i]).T @ w + K[i].T @ r[i]
        else:
            kf[i] = np.zeros(0)
            p[i] = q[i] + A.T @ w
    z, v = [z0] + [None] * N, [None] * N
    for i in range(N):
        v[i] = K[i] @ z[i] + kf[i]
        z[i + 1] = b["A"][i] @ z[i] + b["B"][i] @ v[i] + c[i]
    return z, v, [P[i] @ z[i] + p[i] for i in range(N + 1)]


def _kkt_residual(b, N, z, v, lam):
    rq, rr, rc = [None] * (N + 1), [None] * N, [None] * N
    rq[N] = b["Q"][N] @ z[N] + b["q"][N] - lam[N]
    for i in range(N):
        A, B, Q, M, R = b["A"][i], b["B"][i], b["Q"][i], b["M"][i], b["R"][i]
        rq[i] = Q @ z[i] + M @ v[i] + b["q"][i] + A.T @ lam[i + 1] - lam[i]
        rr[i] = R @ v[i] + M.T @ z[i] + b["r"][i] + B.T @ lam[i + 1]
        rc[i] = A @ z[i] + B @ v[i] + b["c"][i] - z[i + 1]
    return rq, rr, rc


def refinement_errors(pb, dt, passes):
    """Relative (z, v) error against the oracle after 0..passes refinement passes."""
    b, N = _reduced(pb)
    fac = _sqrt_riccati(b, N, dt)
    z, v, lam = _solve(b, N, fac, b["q"], b["r"], b["c"], b["z"][0])
    scale = max(1.0, max(float(np.abs(x).max()) for x in b["z"] + b["v"] if x.size))
    errs = []
    for k in range(passes + 1):
        e = max(float(np.abs(x - y).max()) if x.size else 0.0 for x, y in zip(z + v, b["z"] + b["v"]))
        errs.append(e / scale if np.isfinite(e) else np.inf)
        if k == passes:
            break
        rq, rr, rc = _kkt_residual(b, N, z, v, lam)
        dz, dv, dl = _solve(b, N, fac, rq, rr, rc, np.zeros_like(z[0]))
        z = [x + y for x, y in zip(z, dz)]
        v = [x + y for x, y in zip(v, dv)]
        lam = [x + y for x, y in zip(lam, dl)]
    return errs


def test_fp64_factors_refine_to_the_oracle():
    """The emulated solve itself is sound: FP64 factors reach the oracle's reduced solution."""
    errs = refinement_errors(synth.config("diff_batch", index=0), np.float64, 2)
    assert errs[-1] <= 1e-12, errs


def test_fp32_factors_refine_on_the_well_conditioned_draw():
    errs = refinement_errors(synth.config("diff_batch", index=0), np.float32, 3)
    assert errs[0] > 1e-6, errs  # the FP32 factors are only FP32-accurate
    assert errs[-1] <= 1e-9, errs


@pytest.mark.parametrize("name,index", [("degenerate_n12", 0), ("batched_uneven", 0), ("batched_uneven", 2)])
def test_fp32_factors_do_not_reach_the_tolerance_on_ill_conditioned_workloads(name, index):
    pb = synth.config(name, index=index)
    e32 = refinement_errors(pb, np.float32, 4)
    e64 = refinement_errors(pb, np.float64, 2)
    assert e64[-1] <= 1e-9, e64
    assert not (e32[-1] <= 1e-9), e32
