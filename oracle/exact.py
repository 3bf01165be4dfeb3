"""O1 at full size -- the KKT system solved by sparse LU, refined in extended precision.

TEST INFRASTRUCTURE ONLY.

The plain definition again (Sec. 2 problem; Sec. 7 stationarity and sign
convention), as in ``dense.py``, but assembled sparse so that whole workloads
fit: the KKT matrix of one problem has a few entries per row.  It is factored
once in FP64 (scipy's SuperLU with partial pivoting) and the solution is
refined with residuals accumulated in numpy's ``longdouble`` (64-bit mantissa
on x86-64), which makes it accurate to about the extended unit roundoff times
the conditioning: far below FP64 rounding for the workloads here.

``exact_kkt`` returns that solution rounded to FP64.  Its Sec. 9 residual,
evaluated in FP64, is the residual floor of the problem: no FP64 point can be
expected to reach much below it, whatever the method.  ``residual_scale``
gives the componentwise scale (|K||w| + |b|) of every row, whose product with
the unit roundoff bounds the same floor a priori.

Requires a nonsingular KKT matrix (the constraint Jacobian of full row rank),
which the uneven-batch generator gives generically.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spl


def _index(pb):
    n, m = pb.n, pb.m
    xi = lambda i: i * (n + m)          # noqa: E731  first column of x_i
    ui = lambda i: i * (n + m) + n      # noqa: E731  first column of u_i
    return xi, ui


def kkt_matrix(pb):
    """Sparse KKT matrix [[H, J'], [J, 0]] and right-hand side [-g; b] over
    w = (x_0, u_0, ..., x_{N-1}, u_{N-1}, x_N) and the constraint rows, in order,
    x_0 = s_0 (alpha), dynamics (lambda_{i+1}), mixed rows (mu), state-only rows (eta)."""
    N, n, m = pb.N, pb.n, pb.m
    xi, ui = _index(pb)
    nv = N * (n + m) + n
    po = np.concatenate([[0], np.cumsum(pb.p)]).astype(int)
    qo = np.concatenate([[0], np.cumsum(pb.q)]).astype(int)
    rows, cols, vals = [], [], []

    def put(r0, c0, blk):
        blk = np.asarray(blk, dtype=np.float64)
        if blk.size == 0:
            return
        rr, cc = np.nonzero(np.ones_like(blk, dtype=bool))
        rows.append(rr + r0)
        cols.append(cc + c0)
        vals.append(blk[rr, cc])

    g = np.zeros(nv)
    for i in range(N):
        put(xi(i), xi(i), pb.Q[i]); put(xi(i), ui(i), pb.M[i])
        put(ui(i), xi(i), pb.M[i].T); put(ui(i), ui(i), pb.R[i])
        g[xi(i):xi(i) + n] = pb.qv[i]
        g[ui(i):ui(i) + m] = pb.rv[i]
    put(xi(N), xi(N), pb.Q[N])
    g[xi(N):xi(N) + n] = pb.qv[N]
    # constraint rows J (placed at row offset nv) and their transposes
    nr = n + N * n + int(po[-1]) + int(qo[-1])
    b = np.zeros(nr)
    jr, jc, jv = [], [], []

    def putj(r0, c0, blk):
        blk = np.asarray(blk, dtype=np.float64)
        if blk.size == 0:
            return
        rr, cc = np.nonzero(np.ones_like(blk, dtype=bool))
        jr.append(rr + r0)
        jc.append(cc + c0)
        jv.append(blk[rr, cc])

    r = 0
    putj(r, xi(0), np.eye(n)); b[r:r + n] = pb.s0; r += n
    for i in range(N):
        putj(r, xi(i), pb.A[i]); putj(r, ui(i), pb.B[i]); putj(r, xi(i + 1), -np.eye(n))
        b[r:r + n] = -pb.c[i]
        r += n
    for i in range(N):
        k = int(pb.p[i])
        putj(r, xi(i), pb.C[po[i]:po[i + 1]]); putj(r, ui(i), pb.D[po[i]:po[i + 1]])
        b[r:r + k] = -pb.d[po[i]:po[i + 1]]
        r += k
    for i in range(N + 1):
        k = int(pb.q[i])
        putj(r, xi(i), pb.E[qo[i]:qo[i + 1]])
        b[r:r + k] = -pb.e[qo[i]:qo[i + 1]]
        r += k
    jr, jc, jv = (np.concatenate(a) for a in (jr, jc, jv))
    rows = np.concatenate(rows + [jr + nv, jc])
    cols = np.concatenate(cols + [jc, jr + nv])
    vals = np.concatenate(vals + [jv, jv])
    K = sp.csr_matrix((vals, (rows, cols)), shape=(nv + nr, nv + nr))
    return K, np.concatenate([-g, b]), nv


def _unpack(pb, sol, nv):
    N, n, m = pb.N, pb.n, pb.m
    w, y = sol[:nv], sol[nv:]
    x = np.stack([w[i * (n + m):i * (n + m) + n] for i in range(N + 1)])
    u = np.stack([w[i * (n + m) + n:(i + 1) * (n + m)] for i in range(N)])
    alpha = y[:n].copy()
    lam = np.zeros((N + 1, n))
    lam[1:] = y[n:n + N * n].reshape(N, n)
    lam[0] = -alpha
    P = int(np.sum(pb.p))
    mu = y[n + N * n:n + N * n + P].copy()
    eta = y[n + N * n + P:].copy()
    return dict(x=x, u=u, lam=lam, mu=mu, eta=eta, alpha=alpha)


def solve_refined(K, rhs, passes=6, lu=None):
    """K w = rhs by one FP64 sparse LU and `passes` steps of refinement whose residuals are
    accumulated in extended precision; returns (w in FP64, extended-precision residual norm, lu)."""
    lu = lu or spl.splu(K.tocsc())
    Kl = K.astype(np.longdouble)
    rl = np.asarray(rhs, dtype=np.float64).astype(np.longdouble)
    sl = lu.solve(np.asarray(rhs, dtype=np.float64)).astype(np.longdouble)
    for _ in range(passes):
        r = rl - Kl @ sl
        sl = sl + lu.solve(np.asarray(r, dtype=np.float64)).astype(np.longdouble)
    return np.asarray(sl, dtype=np.float64), float(np.max(np.abs(rl - Kl @ sl))), lu


def exact_kkt(pb, passes=6):
    """The KKT solution, refined with extended-precision residuals and rounded to FP64.
    Also returns 'ext_resid', the infinity norm of the extended-precision residual of the
    unrounded iterate (a measure of how far the refinement got)."""
    K, rhs, nv = kkt_matrix(pb)
    sol, ext, _ = solve_refined(K, rhs, passes)
    out = _unpack(pb, sol, nv)
    out["ext_resid"] = ext
    return out


def residual_scale(pb, sol):
    """Per KKT row, |K||w| + |rhs| at the solution: rounding the solution and evaluating the
    residual in FP64 moves each row by a small multiple of the unit roundoff times this."""
    K, rhs, nv = kkt_matrix(pb)
    N, n, m = pb.N, pb.n, pb.m
    w = np.concatenate([np.concatenate([sol["x"][i], sol["u"][i]]) for i in range(N)] + [sol["x"][N]])
    y = np.concatenate([sol["alpha"], sol["lam"][1:].ravel(), sol["mu"], sol["eta"]])
    return abs(K) @ np.abs(np.concatenate([w, y])) + np.abs(rhs)
