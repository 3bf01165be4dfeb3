"""Parameter gradients of a loss l(x, u) by implicit differentiation of the dense KKT system.

TEST INFRASTRUCTURE ONLY.

The paper has no gradients.  Written from the definition: the primal-dual
solution w(theta) of the problem (Sec. 2) satisfies F(w, theta) = 0, F being
the KKT map of O1 (dense.py) -- stationarity of the Lagrangian of Sec. 7 and
the constraint rows.  By the implicit function theorem
    dl/dtheta = -wb' dF/dtheta,   K' wb = dl/dw,   K = dF/dw,
and K is the dense KKT matrix assembled by dense.py (symmetric).  F is linear
in every matrix and offset, so dF/dtheta for one entry is the pattern that
entry has in K (times the solution) or in the right-hand side; the loops
below read that pattern off the dense row/column index maps of dense.py.
Symmetric parameters (Q_i, R_i) receive the symmetrised gradient.
Pinned against central finite differences of the sequential oracle (O2) in
tests/test_oracle_adjoint.py.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import dense


def _solve_kkt(K, rhs, refine=3):
    sol = sla.lstsq(K, rhs, lapack_driver="gelsd")[0]
    for _ in range(refine):
        sol = sol + sla.lstsq(K, rhs - K @ sol, lapack_driver="gelsd")[0]
    return sol


def implicit_gradients(pb, lx, lu, sparse=False):
    """Gradients of l w.r.t. every problem array, given dl/dx ((N+1) x n) and dl/du (N x m).

    sparse: solve the KKT system and its transpose with the sparse LU of oracle.exact (refined in
    extended precision) instead of the dense least-squares solve -- for full-size problems, whose
    constraint Jacobian must then have full row rank.  The same index maps serve both.
    Returns a dict keyed like the problem fields (A, B, c, C, D, d, E, e, Q, M, R, qv, rv, s0),
    each with the shape of that field."""
    N, n, m = pb.N, pb.n, pb.m
    if sparse:
        from .exact import kkt_matrix, solve_refined
        K, rhs, nv = kkt_matrix(pb)
        nr = K.shape[0] - nv
        sol, _, lu_f = solve_refined(K, rhs)
    else:
        J, b = dense.constraint_matrix(pb)
        H, g = dense.hessian_gradient(pb)
        nv, nr = H.shape[0], J.shape[0]
        K = np.zeros((nv + nr, nv + nr))
        K[:nv, :nv] = H
        K[:nv, nv:] = J.T
        K[nv:, :nv] = J
        sol = _solve_kkt(K, np.concatenate([-g, b]))
    lw = np.zeros(nv + nr)
    for i in range(N + 1):
        lw[dense._xidx(pb, i)] = lx[i]
    for i in range(N):
        lw[dense._uidx(pb, i)] = lu[i]
    adj = solve_refined(K.T.tocsr(), lw, lu=lu_f)[0] if sparse else _solve_kkt(K.T, lw)
    w, y = sol[:nv], sol[nv:]
    wb, yb = adj[:nv], adj[nv:]
    po, qo = dense._offsets(pb)
    X = [w[dense._xidx(pb, i)] for i in range(N + 1)]
    U = [w[dense._uidx(pb, i)] for i in range(N)]
    Xb = [wb[dense._xidx(pb, i)] for i in range(N + 1)]
    Ub = [wb[dense._uidx(pb, i)] for i in range(N)]
    # multiplier rows of the dense system: alpha | dynamics of stage i (lambda_{i+1}) | mixed | state-only
    ya, yba = y[:n], yb[:n]
    Lam = [y[n + i * n:n + (i + 1) * n] for i in range(N)]
    Lamb = [yb[n + i * n:n + (i + 1) * n] for i in range(N)]
    o = n + N * n
    Mu, Mub = y[o:o + po[-1]], yb[o:o + po[-1]]
    Eta, Etab = y[o + po[-1]:], yb[o + po[-1]:]
    G = {k: np.zeros_like(np.asarray(getattr(pb, k), dtype=float)) for k in
         ("A", "B", "c", "C", "D", "d", "E", "e", "Q", "M", "R", "qv", "rv", "s0")}
    for i in range(N):
        # dynamics row of stage i: A x_i + B u_i - x_{i+1} = -c_i, multiplier lambda_{i+1};
        # A enters K at (dyn_i, x_i) and (x_i, dyn_i): -wb' dF/dA[j,k] = -(yb_j x_k + xb_k y_j)
        G["A"][i] = -(np.outer(Lamb[i], X[i]) + np.outer(Lam[i], Xb[i]))
        G["B"][i] = -(np.outer(Lamb[i], U[i]) + np.outer(Lam[i], Ub[i]))
        G["c"][i] = -Lamb[i]                                   # rhs -c_i
        G["M"][i] = -(np.outer(Xb[i], U[i]) + np.outer(X[i], Ub[i]))
        GQ = -np.outer(Xb[i], X[i])
        G["Q"][i] = 0.5 * (GQ + GQ.T)
        GR = -np.outer(Ub[i], U[i])
        G["R"][i] = 0.5 * (GR + GR.T)
        G["qv"][i] = -Xb[i]
        G["rv"][i] = -Ub[i]
        sl = slice(po[i], po[i + 1])
        G["C"][sl] = -(np.outer(Mub[sl], X[i]) + np.outer(Mu[sl], Xb[i]))
        G["D"][sl] = -(np.outer(Mub[sl], U[i]) + np.outer(Mu[sl], Ub[i]))
        G["d"][sl] = -Mub[sl]
    GQ = -np.outer(Xb[N], X[N])
    G["Q"][N] = 0.5 * (GQ + GQ.T)
    G["qv"][N] = -Xb[N]
    for i in range(N + 1):
        sl = slice(qo[i], qo[i + 1])
        G["E"][sl] = -(np.outer(Etab[sl], X[i]) + np.outer(Eta[sl], Xb[i]))
        G["e"][sl] = -Etab[sl]
    G["s0"] = yba.copy()                                       # rhs +s_0 in the x_0 row
    return G
