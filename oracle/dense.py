"""O1 -- the plain definition, with numpy/scipy as the only machinery.

TEST INFRASTRUCTURE ONLY.

Under the convexity assumptions (Sec. 2, eq. convexity) with Q_i, R_i
positive definite, the primal solution of the problem (Sec. 2, eq. problem)
is the unique minimiser of a convex QP, and its KKT multipliers are any
solution of the stationarity equations (Sec. 7, eqs. stage-stationarity,
terminal-stationarity).  This module assembles the whole KKT system

        [ H   J^T ] [ w ]   [ -g ]
        [ J   0   ] [ y ] = [  b ]

over w = (x_0, u_0, x_1, u_1, ..., x_{N-1}, u_{N-1}, x_N) with constraint rows,
in order: x_0 = s_0 (multiplier alpha), dynamics A x_i + B u_i - x_{i+1} = -c_i
(multiplier lambda_{i+1}), mixed rows C x + D u = -d (mu), state-only rows
E x = -e (eta) -- the Lagrangian sign convention of Sec. 7 -- and solves it by
SVD least squares.  The least-squares minimum-norm solution has the unique
primal part and the multiplier of least norm, i.e. the projection of every
valid multiplier onto range(J).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def _offsets(pb):
    po = np.concatenate([[0], np.cumsum(pb.p)]).astype(int)
    qo = np.concatenate([[0], np.cumsum(pb.q)]).astype(int)
    return po, qo


def _xidx(pb, i):
    s = i * (pb.n + pb.m)
    return slice(s, s + pb.n)


def _uidx(pb, i):
    s = i * (pb.n + pb.m) + pb.n
    return slice(s, s + pb.m)


def constraint_matrix(pb):
    """(J, b) with J w = b, rows ordered as in the module docstring."""
    N, n, m = pb.N, pb.n, pb.m
    po, qo = _offsets(pb)
    nv = N * (n + m) + n
    rows = n + N * n + int(po[-1]) + int(qo[-1])
    J = np.zeros((rows, nv))
    b = np.zeros(rows)
    r = 0
    J[r:r + n, _xidx(pb, 0)] = np.eye(n); b[r:r + n] = pb.s0; r += n
    for i in range(N):
        J[r:r + n, _xidx(pb, i)] = pb.A[i]
        J[r:r + n, _uidx(pb, i)] = pb.B[i]
        J[r:r + n, _xidx(pb, i + 1)] = -np.eye(n)
        b[r:r + n] = -pb.c[i]
        r += n
    for i in range(N):
        k = pb.p[i]
        J[r:r + k, _xidx(pb, i)] = pb.C[po[i]:po[i + 1]]
        J[r:r + k, _uidx(pb, i)] = pb.D[po[i]:po[i + 1]]
        b[r:r + k] = -pb.d[po[i]:po[i + 1]]
        r += k
    for i in range(N + 1):
        k = pb.q[i]
        J[r:r + k, _xidx(pb, i)] = pb.E[qo[i]:qo[i + 1]]
        b[r:r + k] = -pb.e[qo[i]:qo[i + 1]]
        r += k
    return J, b


def hessian_gradient(pb):
    N, n, m = pb.N, pb.n, pb.m
    nv = N * (n + m) + n
    H = np.zeros((nv, nv))
    g = np.zeros(nv)
    for i in range(N):
        xi, ui = _xidx(pb, i), _uidx(pb, i)
        H[xi, xi] = pb.Q[i]
        H[xi, ui] = pb.M[i]
        H[ui, xi] = pb.M[i].T
        H[ui, ui] = pb.R[i]
        g[xi] = pb.qv[i]
        g[ui] = pb.rv[i]
    xN = _xidx(pb, N)
    H[xN, xN] = pb.Q[N]
    g[xN] = pb.qv[N]
    return H, g


def objective(pb, x, u):
    """Original objective (Sec. 2, eqs. stage-cost and problem)."""
    f = 0.0
    for i in range(pb.N):
        f += 0.5 * x[i] @ pb.Q[i] @ x[i] + x[i] @ pb.M[i] @ u[i] + 0.5 * u[i] @ pb.R[i] @ u[i]
        f += pb.qv[i] @ x[i] + pb.rv[i] @ u[i]
    f += 0.5 * x[pb.N] @ pb.Q[pb.N] @ x[pb.N] + pb.qv[pb.N] @ x[pb.N]
    return f


def dense_kkt(pb, refine=3):
    """Solve the whole KKT system.  Returns a dict with x, u, lam (lambda_0 = -alpha),
    mu, eta, alpha, the rank of J and its row count."""
    N, n, m = pb.N, pb.n, pb.m
    J, b = constraint_matrix(pb)
    H, g = hessian_gradient(pb)
    nv, nr = H.shape[0], J.shape[0]
    K = np.zeros((nv + nr, nv + nr))
    K[:nv, :nv] = H
    K[:nv, nv:] = J.T
    K[nv:, :nv] = J
    rhs = np.concatenate([-g, b])
    sol, _, rank_k, _ = sla.lstsq(K, rhs, lapack_driver="gelsd")
    # classical iterative refinement: the KKT matrix of these instances reaches
    # condition numbers near 1e9, where one SVD solve keeps only ~7 digits
    for _ in range(refine):
        sol = sol + sla.lstsq(K, rhs - K @ sol, lapack_driver="gelsd")[0]
    w, y = sol[:nv], sol[nv:]
    x = np.stack([w[_xidx(pb, i)] for i in range(N + 1)])
    u = np.stack([w[_uidx(pb, i)] for i in range(N)]) if N else np.zeros((0, m))
    po, qo = _offsets(pb)
    alpha = y[:n]
    lam = np.zeros((N + 1, n))
    lam[0] = -alpha
    lam[1:] = y[n:n + N * n].reshape(N, n)
    o = n + N * n
    mu = y[o:o + po[-1]]
    eta = y[o + po[-1]:]
    return dict(x=x, u=u, lam=lam, mu=mu, eta=eta, alpha=alpha,
                rank_J=int(np.linalg.matrix_rank(J)), rows_J=nr, kkt_rank=int(rank_k),
                J=J, H=H, g=g)


def multiplier_vector(pb, lam, mu, eta, alpha):
    """Stack multipliers in the dense row order (alpha, lambda_1..N, mu, eta)."""
    return np.concatenate([alpha, lam[1:].ravel(), mu, eta])


def brute_suffix_domain(pb, i, tol=1e-9):
    """X_i of Thm 3 by brute force: stack every constraint from stage i to the
    terminal stage over (x_i, u_i, x_{i+1}, ..., x_N) and project out all but
    x_i with an SVD null space (Lemma 1).  Returns (H, h) with orthonormal rows
    (possibly zero rows) and a flag telling whether the system is consistent."""
    N, n, m = pb.N, pb.n, pb.m
    po, qo = _offsets(pb)
    nvar = (N - i) * (n + m) + n
    def xs(k):
        s = (k - i) * (n + m)
        return slice(s, s + n)
    def us(k):
        s = (k - i) * (n + m) + n
        return slice(s, s + m)
    rows = []
    rhs = []
    for k in range(i, N):
        Rk = np.zeros((n, nvar)); Rk[:, xs(k)] = pb.A[k]; Rk[:, us(k)] = pb.B[k]; Rk[:, xs(k + 1)] = -np.eye(n)
        rows.append(Rk); rhs.append(pb.c[k])
        pk = pb.p[k]
        if pk:
            Rk = np.zeros((pk, nvar)); Rk[:, xs(k)] = pb.C[po[k]:po[k + 1]]; Rk[:, us(k)] = pb.D[po[k]:po[k + 1]]
            rows.append(Rk); rhs.append(pb.d[po[k]:po[k + 1]])
    for k in range(i, N + 1):
        qk = pb.q[k]
        if qk:
            Rk = np.zeros((qk, nvar)); Rk[:, xs(k)] = pb.E[qo[k]:qo[k + 1]]
            rows.append(Rk); rhs.append(pb.e[qo[k]:qo[k + 1]])
    if not rows:
        return np.zeros((0, n)), np.zeros(0), True
    G = np.vstack(rows)
    g = np.concatenate(rhs)
    Gx, Gw = G[:, :n], G[:, n:]
    # W: orthonormal basis of null(Gw^T) = range(Gw)^perp
    if Gw.shape[1] == 0:
        W = np.eye(G.shape[0])
    else:
        U, s, _ = np.linalg.svd(Gw, full_matrices=True)
        rk = int(np.sum(s > tol * max(1.0, s[0] if s.size else 0.0)))
        W = U[:, rk:]
    Hx = W.T @ Gx
    hx = W.T @ g
    # compress to an orthonormal row basis
    if Hx.shape[0] == 0:
        return np.zeros((0, n)), np.zeros(0), True
    U2, s2, Vt2 = np.linalg.svd(Hx, full_matrices=True)
    rk2 = int(np.sum(s2 > tol * max(1.0, s2[0] if s2.size else 0.0)))
    Hc = Vt2[:rk2]
    hc = (U2[:, :rk2].T @ hx) / s2[:rk2]
    resid = U2[:, rk2:].T @ hx
    consistent = bool(np.all(np.abs(resid) <= 1e-8 * max(1.0, np.max(np.abs(hx)) if hx.size else 1.0)))
    return Hc, hc, consistent
