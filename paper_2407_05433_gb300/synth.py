"""Seeded synthetic ECLQR instances.

This module only draws problem data; it contains none of the reduction's
arithmetic.  Both the CUDA path (through the tests and the benchmark) and the
CPU oracle receive the same arrays produced here.

Problem statement (Sec. 2, eq. problem):

    min  sum_i l_i(x_i, u_i) + 1/2 x_N^T Q_N x_N + q_N^T x_N
    s.t. x_0 = s_0
         x_{i+1} = A_i x_i + B_i u_i + c_i        i = 0..N-1
         C_i x_i + D_i u_i + d_i = 0               i = 0..N-1
         E_i x_i + e_i = 0                         i = 0..N

with l_i(x, u) = 1/2 x^T Q_i x + x^T M_i u + 1/2 u^T R_i u + q_i^T x + r_i^T u
(eq. stage-cost).  State and control dimensions are uniform within one
problem; constraint row counts p_i (mixed) and q_i (state-only) vary per stage.
Stage-varying n_i, m_i enter through pack_varying (zero padding to the largest
ones, which leaves the solution on the original coordinates unchanged).

Packed layout (row-major, stage after stage), shared by every consumer:
    A (N,n,n)  B (N,n,m)  c (N,n)
    C (sum p, n)  D (sum p, m)  d (sum p)       rows of stage i follow stage i-1
    E (sum q, n)  e (sum q)                     stages 0..N (terminal last)
    Q (N+1,n,n)  qv (N+1,n)                     block N is Q_N, q_N
    M (N,n,m)  R (N,m,m)  rv (N,m)
    s0 (n)

Feasibility is by construction: a random trajectory (x*, u*) is drawn first and
c, d, e are set so that it satisfies every constraint, with s_0 = x*_0.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

__all__ = ["ECLQRProblem", "make_problem", "config", "CONFIG_NAMES", "random_spd", "pack_varying",
           "unpack_varying"]


@dataclass
class ECLQRProblem:
    N: int
    n: int
    m: int
    p: np.ndarray
    q: np.ndarray
    A: np.ndarray
    B: np.ndarray
    c: np.ndarray
    C: np.ndarray
    D: np.ndarray
    d: np.ndarray
    E: np.ndarray
    e: np.ndarray
    Q: np.ndarray
    M: np.ndarray
    R: np.ndarray
    qv: np.ndarray
    rv: np.ndarray
    s0: np.ndarray
    x_star: np.ndarray = field(default=None, repr=False)
    u_star: np.ndarray = field(default=None, repr=False)

    @property
    def stages(self) -> int:
        return self.N

    def copy(self) -> "ECLQRProblem":
        kw = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in self.__dict__.items()}
        return ECLQRProblem(**kw)


def random_spd(rng, k, eps=1e-3):
    L = rng.standard_normal((k, k))
    return L @ L.T + eps * np.eye(k)


def _orthogonal(rng, n):
    G = rng.standard_normal((n, n))
    Qf, Rf = np.linalg.qr(G)
    return Qf * np.sign(np.diag(Rf))[None, :]


def make_problem(seed, N, n, m, p, q, *, a_mode="perturbed", degenerate_frac=0.0,
                 cross=False, zero_D_rows=None, dup_rows=None):
    """Draw one feasible instance.

    p: int or sequence of N ints (mixed rows per stage); q: int or sequence of
    N+1 ints (state-only rows, q[N] is the terminal row count).
    a_mode: "perturbed" (A = I + 0.1 randn) or "orthogonal" (spectral radius 1).
    degenerate_frac: fraction of stages given duplicated mixed rows or rows
    with D = 0 (state-only rows written as mixed rows).
    cross: draw nonzero M_i (then Q, M, R are drawn jointly PSD).
    """
    rng = np.random.default_rng(seed)
    p = np.full(N, p, dtype=np.int32) if np.isscalar(p) else np.asarray(p, dtype=np.int32).copy()
    q = np.full(N + 1, q, dtype=np.int32) if np.isscalar(q) else np.asarray(q, dtype=np.int32).copy()
    assert p.shape == (N,) and q.shape == (N + 1,)
    # Draws come in a fixed order; a generator fills an array of draws in the same order as the
    # same number of one-block calls, so whole arrays are drawn at once.
    if a_mode == "perturbed":
        A = np.eye(n)[None] + 0.1 * rng.standard_normal((N, n, n))
    elif a_mode == "orthogonal":
        A = np.stack([_orthogonal(rng, n) for _ in range(N)])
    else:
        raise ValueError(a_mode)
    B = rng.standard_normal((N, n, m))
    if cross:
        Hs = [random_spd(rng, n + m) for _ in range(N)]
        Q = np.stack([Hk[:n, :n] for Hk in Hs] + [random_spd(rng, n)])
        M = np.stack([Hk[:n, n:] for Hk in Hs])
        R = np.stack([Hk[n:, n:] for Hk in Hs])
    else:
        LQ = rng.standard_normal((N + 1, n, n))
        Q = LQ @ LQ.transpose(0, 2, 1) + 1e-3 * np.eye(n)[None]
        LR = rng.standard_normal((N, m, m))
        R = LR @ LR.transpose(0, 2, 1) + 1e-3 * np.eye(m)[None]
        M = np.zeros((N, n, m))
    qv = rng.standard_normal((N + 1, n))
    rv = rng.standard_normal((N, m))
    P = int(p.sum())
    Cm = rng.standard_normal((P, n))
    Dm = rng.standard_normal((P, m))
    Em = rng.standard_normal((int(q.sum()), n))
    # structural degeneracy (duplicated rows, D = 0 rows)
    po = np.concatenate([[0], np.cumsum(p)])
    if degenerate_frac > 0:
        ndeg = int(round(degenerate_frac * N))
        stages = rng.choice(N, size=ndeg, replace=False)
        kinds = rng.integers(0, 2, size=ndeg)
        for s, kind in zip(stages, kinds):
            lo, hi = po[s], po[s + 1]
            if hi - lo == 0:
                continue
            if kind == 0 and hi - lo >= 2:
                j = rng.integers(lo, hi - 1)
                Cm[j + 1] = Cm[j]
                Dm[j + 1] = Dm[j]
            else:
                k = max(1, (hi - lo + 1) // 2)
                rows = rng.choice(np.arange(lo, hi), size=k, replace=False)
                Dm[rows] = 0.0
    if zero_D_rows is not None:
        Dm[np.asarray(zero_D_rows)] = 0.0
    if dup_rows is not None:
        for j, k in dup_rows:
            Cm[k] = Cm[j]
            Dm[k] = Dm[j]
    # feasible trajectory
    xs = rng.standard_normal((N + 1, n))
    us = rng.standard_normal((N, m))
    c = xs[1:] - np.einsum("ijk,ik->ij", A, xs[:-1]) - np.einsum("ijk,ik->ij", B, us)
    stage_of_row = np.repeat(np.arange(N), p)
    d = -(np.einsum("rj,rj->r", Cm, xs[stage_of_row]) + np.einsum("rj,rj->r", Dm, us[stage_of_row]))
    e = -np.einsum("rj,rj->r", Em, xs[np.repeat(np.arange(N + 1), q)])
    return ECLQRProblem(N=N, n=n, m=m, p=p, q=q, A=A, B=B, c=c, C=Cm, D=Dm, d=d,
                        E=Em, e=e, Q=Q, M=M, R=R, qv=qv, rv=rv, s0=xs[0].copy(),
                        x_star=xs, u_star=us)


def pack_varying(A, B, c, C, D, d, E, e, Q, M, R, qv, rv, s0):
    """One problem with stage-varying dimensions (Sec. 2: x_i in R^{n_i}, u_i in R^{m_i}) in the packed
    per-problem layout, by zero padding to n = max n_i and m = max m_i.

    Per-stage lists: A[i] (n_{i+1}, n_i), B[i] (n_{i+1}, m_i), c[i] (n_{i+1},), C[i] (p_i, n_i),
    D[i] (p_i, m_i), d[i] (p_i,), M[i] (n_i, m_i), R[i] (m_i, m_i), rv[i] (m_i,) for i < N;
    E[i] (q_i, n_i), e[i] (q_i,), Q[i] (n_i, n_i), qv[i] (n_i,) for i <= N; s0 (n_0,).
    Padded coordinates get zero rows and columns everywhere and identity blocks in Q and R: the padded
    states stay 0 through the dynamics, the padded controls sit at their minimum 0, and the multipliers
    of the padded rows are 0, so the solution on the original coordinates is unchanged.
    Returns (problem, (n_i, m_i)); unpack_varying cuts a solution back to the original shapes."""
    N = len(A)
    ni = [Q[i].shape[0] for i in range(N + 1)]
    mi = [R[i].shape[0] for i in range(N)]
    n, m = max(ni), max(mi)

    def put(block, shape):
        out = np.zeros(shape)
        block = np.asarray(block, dtype=np.float64)
        out[tuple(slice(0, k) for k in block.shape)] = block
        return out

    def eye_pad(block, k):
        out = put(block, (k, k))
        for j in range(np.asarray(block).shape[0], k):
            out[j, j] = 1.0
        return out

    p = np.array([np.asarray(d[i]).size for i in range(N)], dtype=np.int32)
    q = np.array([np.asarray(e[i]).size for i in range(N + 1)], dtype=np.int32)
    pb = ECLQRProblem(
        N=N, n=n, m=m, p=p, q=q,
        A=np.stack([put(A[i], (n, n)) for i in range(N)]),
        B=np.stack([put(B[i], (n, m)) for i in range(N)]),
        c=np.stack([put(c[i], (n,)) for i in range(N)]),
        C=np.concatenate([put(C[i], (p[i], n)) for i in range(N)]),
        D=np.concatenate([put(D[i], (p[i], m)) for i in range(N)]),
        d=np.concatenate([np.asarray(d[i], dtype=np.float64).reshape(-1) for i in range(N)]),
        E=np.concatenate([put(E[i], (q[i], n)) for i in range(N + 1)]),
        e=np.concatenate([np.asarray(e[i], dtype=np.float64).reshape(-1) for i in range(N + 1)]),
        Q=np.stack([eye_pad(Q[i], n) for i in range(N + 1)]),
        M=np.stack([put(M[i], (n, m)) for i in range(N)]),
        R=np.stack([eye_pad(R[i], m) for i in range(N)]),
        qv=np.stack([put(qv[i], (n,)) for i in range(N + 1)]),
        rv=np.stack([put(rv[i], (m,)) for i in range(N)]),
        s0=put(s0, (n,)))
    return pb, (ni, mi)


def unpack_varying(dims, x, u, lam, alpha):
    """Per-stage x_i (n_i), u_i (m_i), lambda_i (n_i) and alpha (n_0) of a pack_varying problem's solution;
    mu and eta keep their packed order (the row counts were not padded)."""
    ni, mi = dims
    return ([np.asarray(x[i])[:ni[i]] for i in range(len(ni))], [np.asarray(u[i])[:mi[i]] for i in range(len(mi))],
            [np.asarray(lam[i])[:ni[i]] for i in range(len(ni))], np.asarray(alpha)[:ni[0]])


CONFIG_NAMES = ("single_n4", "degenerate_n12", "long_n16", "batched_uneven", "diff_batch", "table1",
                "mixed_only_n12")


def config(name, seed=0, N=None, index=0):
    """Instances with the shapes and structure of the five benchmark workloads.

    single_n4       N=64, n=4, m=2, one mixed row per stage, rank-2 terminal rows.
    degenerate_n12  N=1024, n=12, m=6, mixed rows U{0..8} per stage, 20% of
                    stages with duplicated or D=0 rows, full-rank terminal.
    long_n16        N=65536, n=16, m=8, 4 mixed rows per stage, terminal of
                    rank 8, A orthogonal (spectral radius 1).
    batched_uneven  problem `index` of the batch: N ~ U[32,512],
                    n in {8,12,16,24}, m = n/2, mixed rows U{0..m},
                    terminal rows U{0..n/2}; seed = seed + index.
    diff_batch      problem `index`: N=256, n=16, m=8, 4 mixed rows,
                    4 terminal rows; seed = seed + index.
    table1          the paper's Table 1 shape: n=8, m=4, two state-only rows
                    per nonterminal stage, no mixed or terminal rows.
    mixed_only_n12  N=1024, n=12, m=6, mixed rows U{0..4} per stage, no
                    state-only or terminal rows: every D_i (p_i x m, randn,
                    p_i < m) is wide with full row rank, so X_i = R^n for all
                    i (the shortcut case of Sec. 6).  Square D_i are left out:
                    their occasional ill-conditioning puts even the oracle's
                    residual above 1e-9 over 1024 unconstrained stages.
    `N` overrides the horizon (shrunk instances of the same generator).
    """
    if name == "single_n4":
        N = 64 if N is None else N
        q = np.zeros(N + 1, dtype=np.int32); q[N] = 2
        return make_problem(seed, N, 4, 2, 1, q)
    if name == "degenerate_n12":
        N = 1024 if N is None else N
        rng = np.random.default_rng(10_000 + seed)
        p = rng.integers(0, 9, size=N)
        q = np.zeros(N + 1, dtype=np.int32); q[N] = 12
        return make_problem(seed, N, 12, 6, p, q, degenerate_frac=0.2)
    if name == "long_n16":
        N = 65536 if N is None else N
        q = np.zeros(N + 1, dtype=np.int32); q[N] = 8
        return make_problem(seed, N, 16, 8, 4, q, a_mode="orthogonal")
    if name == "batched_uneven":
        s = seed + index
        rng = np.random.default_rng(20_000 + s)
        NN = int(rng.integers(32, 513)) if N is None else N
        n = int(rng.choice([8, 12, 16, 24]))
        m = n // 2
        p = rng.integers(0, m + 1, size=NN)
        q = np.zeros(NN + 1, dtype=np.int32); q[NN] = int(rng.integers(0, n // 2 + 1))
        return make_problem(s, NN, n, m, p, q)
    if name == "diff_batch":
        N = 256 if N is None else N
        q = np.zeros(N + 1, dtype=np.int32); q[N] = 4
        return make_problem(seed + index, N, 16, 8, 4, q)
    if name == "mixed_only_n12":
        N = 1024 if N is None else N
        rng = np.random.default_rng(30_000 + seed)
        p = rng.integers(0, 5, size=N)
        return make_problem(seed, N, 12, 6, p, np.zeros(N + 1, dtype=np.int32))
    if name == "table1":
        N = 1024 if N is None else N
        q = np.full(N + 1, 2, dtype=np.int32); q[N] = 0
        return make_problem(seed, N, 8, 4, 0, q)
    raise KeyError(name)
