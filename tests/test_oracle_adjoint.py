"""The dense implicit gradient of the oracle against central finite differences
of the sequential oracle (O2), parameter block by parameter block.

The loss is the differentiable-batch configuration's:
l = sum_i ||x_i - x_ref,i||^2 + sum_i ||u_i||^2.  Symmetric Q_i, R_i are
perturbed symmetrically (the gradient is the symmetrised one)."""
import numpy as np
import pytest

import oracle
from oracle.adjoint import implicit_gradients
from paper_2407_05433_gb300 import synth

H = 1e-6
FIELDS = ("A", "B", "c", "C", "D", "d", "E", "e", "Q", "M", "R", "qv", "rv", "s0")


def loss_and_grads(pb, xref):
    s = oracle.solve(pb, refine=3)
    assert s.ok
    lx = 2.0 * (s.x - xref)
    lu = 2.0 * s.u
    return float(np.sum((s.x - xref) ** 2) + np.sum(s.u ** 2)), lx, lu


def loss(pb, xref):
    return loss_and_grads(pb, xref)[0]


def perturbed(pb, field, idx, h):
    q = pb.copy()
    arr = np.array(getattr(q, field), dtype=float, copy=True)
    arr[idx] += h
    if field in ("Q", "R") and idx[-1] != idx[-2]:
        j = tuple(idx[:-2]) + (idx[-1], idx[-2])
        arr[j] += h
    setattr(q, field, arr)
    return q


@pytest.mark.parametrize("cross", [False, True])
def test_dense_implicit_gradient_matches_finite_differences(cross):
    q = np.zeros(6, np.int32); q[3] = 1; q[5] = 2
    pb = synth.make_problem(41, 5, 3, 2, 1, q, cross=cross)
    rng = np.random.default_rng(7)
    xref = rng.standard_normal((pb.N + 1, pb.n))
    _, lx, lu = loss_and_grads(pb, xref)
    G = implicit_gradients(pb, lx, lu)
    for field in FIELDS:
        arr = np.asarray(getattr(pb, field))
        if arr.size == 0:
            continue
        picks = rng.choice(arr.size, size=min(4, arr.size), replace=False)
        for flat in picks:
            idx = np.unravel_index(flat, arr.shape)
            fd = (loss(perturbed(pb, field, idx, H), xref) - loss(perturbed(pb, field, idx, -H), xref)) / (2 * H)
            g = G[field][idx]
            if field in ("Q", "R") and idx[-1] != idx[-2]:
                g = g + G[field][tuple(idx[:-2]) + (idx[-1], idx[-2])]
            assert abs(fd - g) <= 2e-6 * max(1.0, abs(g)), (field, idx, fd, g)


def test_gradient_of_linear_cost_is_the_solution():
    """Special case by hand: for l = qv_k . x_k-independent part, dl/dqv = -xb where xb
    solves the adjoint; with l = x_N[0] (lx = e_0 at stage N), dl/ds0 must equal the
    sensitivity of x_N[0] to s0 -- checked against the solution's exact linearity in s0."""
    pb = synth.make_problem(43, 4, 3, 2, 0, 0)
    lx = np.zeros((pb.N + 1, pb.n)); lx[pb.N, 0] = 1.0
    lu = np.zeros((pb.N, pb.m))
    G = implicit_gradients(pb, lx, lu)
    base = oracle.solve(pb, refine=3).x[pb.N, 0]
    for k in range(pb.n):
        q = pb.copy(); q.s0 = q.s0.copy(); q.s0[k] += 1.0
        # without state constraints x depends affinely on s0, so a unit step is exact
        assert abs((oracle.solve(q, refine=3).x[pb.N, 0] - base) - G["s0"][k]) < 1e-9


@pytest.mark.parametrize("index", [0, 1])
def test_sparse_implicit_gradient_matches_dense(index):
    """The sparse form of the implicit gradient (oracle.exact's LU, for full-size problems) against the
    dense least-squares form, on shrunk differentiable-batch draws."""
    pb = synth.config("diff_batch", index=index, N=12)
    rng = np.random.default_rng(index)
    lx, lu = rng.standard_normal((pb.N + 1, pb.n)), rng.standard_normal((pb.N, pb.m))
    a, b = implicit_gradients(pb, lx, lu), implicit_gradients(pb, lx, lu, sparse=True)
    for k in FIELDS:
        ref = np.asarray(a[k])
        if ref.size:
            assert np.max(np.abs(np.asarray(b[k]) - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref))), k
