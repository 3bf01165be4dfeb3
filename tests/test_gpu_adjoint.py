"""Gradients through the CUDA path (autograd over eclqr_param_grads) against the
oracle's dense implicit gradient and against central finite differences of the
CUDA solve itself (symmetric Q_i, R_i only in the dense comparison: a
single-entry step leaves the symmetric parameter space).  Loss of the differentiable-batch configuration:
l = sum ||x_i - x_ref,i||^2 + sum ||u_i||^2."""
import numpy as np
import pytest

import oracle
from oracle.adjoint import implicit_gradients
from paper_2407_05433_gb300 import eclqr, synth

pytestmark = pytest.mark.gpu
FIELDS = ("A", "B", "c", "C", "D", "d", "E", "e", "Q", "M", "R", "qv", "rv", "s0")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2407_05433_gb300 import build as b
    b.build()
    eclqr.load()


def _problems():
    q = np.zeros(8, np.int32); q[4] = 1; q[7] = 2
    return [synth.config("diff_batch", index=0, N=8), synth.config("diff_batch", index=1, N=6),
            synth.make_problem(45, 7, 5, 3, 2, q, cross=True)]


def _setup():
    import torch
    from paper_2407_05433_gb300 import autograd as ag
    pbs = _problems()
    batch = eclqr.Batch(pbs)
    rng = np.random.default_rng(3)
    xrefs = [rng.standard_normal((pb.N + 1, pb.n)) for pb in pbs]
    xref = torch.from_numpy(np.concatenate([x.ravel() for x in xrefs])).to(batch.device)
    params = ag.batch_params(batch)
    return torch, ag, pbs, batch, xrefs, xref, params


def _loss(torch, ag, batch, xref, params):
    x, u = ag.solve(batch, *params)
    return ((x - xref) ** 2).sum() + (u ** 2).sum()


def test_autograd_matches_dense_implicit_gradient():
    torch, ag, pbs, batch, xrefs, xref, params = _setup()
    try:
        loss = _loss(torch, ag, batch, xref, params)
        loss.backward()
        got = {k: p.grad.cpu().numpy() for k, p in zip(ag.PARAM_KEYS, params)}
        exp = {k: [] for k in FIELDS}
        for pb, xr in zip(pbs, xrefs):
            s = oracle.dense_kkt(pb)
            G = implicit_gradients(pb, 2.0 * (s["x"] - xr), 2.0 * s["u"])
            for k in FIELDS:
                exp[k].append(np.asarray(G[k]).ravel())
        for k in FIELDS:
            e = np.concatenate(exp[k])
            if e.size == 0:
                continue
            err = np.max(np.abs(got[k][:e.size] - e)) / max(1.0, np.max(np.abs(e)))
            assert err <= 1e-8, (k, err)
    finally:
        batch.close()


def test_autograd_matches_finite_differences_of_the_cuda_solve():
    torch, ag, pbs, batch, xrefs, xref, params = _setup()
    try:
        loss = _loss(torch, ag, batch, xref, params)
        loss.backward()
        rng = np.random.default_rng(11)
        h = 1e-6
        for k in ("A", "B", "c", "C", "D", "M", "E", "e", "qv", "rv", "s0"):
            p = params[ag.PARAM_KEYS.index(k)]
            for flat in rng.choice(p.numel(), size=3, replace=False):
                def f(delta):
                    q = [t.detach().clone() for t in params]
                    q[ag.PARAM_KEYS.index(k)][flat] += delta
                    with torch.no_grad():
                        return float(_loss(torch, ag, batch, xref, q))
                fd = (f(h) - f(-h)) / (2 * h)
                g = float(p.grad[flat])
                assert abs(fd - g) <= 1e-5 * max(1.0, abs(g)), (k, int(flat), fd, g)
    finally:
        batch.close()


def test_adjoint_on_reused_factors_matches_rebuilt_adjoint():
    """eclqr_set_costs + solve (no new build) gives the gradients of a full adjoint rebuild."""
    torch, ag, pbs, batch, xrefs, xref, params = _setup()
    try:
        grads = {}
        for reuse in (True, False):
            ag.ECLQRSolve.reuse_factors = reuse
            ps = [p.detach().clone().requires_grad_(True) for p in params]
            _loss(torch, ag, batch, xref, ps).backward()
            grads[reuse] = [p.grad.clone() for p in ps]
        for k, a, b in zip(ag.PARAM_KEYS, grads[True], grads[False]):
            if b.numel() == 0:
                continue
            err = float((a - b).abs().max()) / max(1.0, float(b.abs().max()))
            assert err <= 1e-9, (k, err)
    finally:
        ag.ECLQRSolve.reuse_factors = True
        batch.close()


def test_batch_refuses_its_own_calls_after_autograd_until_rebuilt():
    """autograd builds the handle on copies of the data (and backward points it at the adjoint's
    arrays), which are freed with the graph: the Batch's own solve and residual refuse to run on
    those pointers, and after build() they give the oracle's solution again."""
    import gc
    torch, ag, pbs, batch, xrefs, xref, params = _setup()
    try:
        _loss(torch, ag, batch, xref, params).backward()
        del params
        gc.collect()
        torch.cuda.empty_cache()
        for call in (batch.solve, batch.multipliers, batch.residual, batch.refine):
            with pytest.raises(RuntimeError, match="build"):
                call()
        batch.run()
        for pb, r in zip(pbs, batch.results()):
            s = oracle.solve(pb)
            assert r["status"] == 0 and r["resid"] <= 1e-9
            for k in ("x", "u", "lam", "mu", "eta", "alpha"):
                ref = getattr(s, k)
                if ref.size:
                    assert np.max(np.abs(r[k] - ref)) / max(1.0, np.max(np.abs(ref))) <= 1e-9, k
    finally:
        batch.close()


def _config5(torch, ag, count=1024):
    pbs = [synth.config("diff_batch", index=j) for j in range(count)]
    batch = eclqr.Batch(pbs)
    rng = np.random.default_rng(5)
    xrefs = [rng.standard_normal((pb.N + 1, pb.n)) for pb in pbs]
    xref = torch.from_numpy(np.concatenate([x.ravel() for x in xrefs])).to(batch.device)
    return pbs, batch, xrefs, xref


def _slices(pbs, j):
    """Packed offsets of problem j's block in every field (all problems share one structure)."""
    pb = pbs[j]
    return {k: slice(j * np.asarray(getattr(pb, k)).size, (j + 1) * np.asarray(getattr(pb, k)).size) for k in FIELDS}


SAMPLED = (0, 345, 1023)


def test_config5_full_batch_against_the_implicit_gradient():
    """The differentiable batch at its full size (1024 problems, N = 256, n = 16, m = 8): the gradient of
    l = sum ||x - x_ref||^2 + ||u||^2 with respect to every field, on three sampled problems, against
    the oracle's implicit gradient of the same loss (sparse KKT solves refined in extended precision),
    every block at 1e-9 relative to its largest entry."""
    import torch
    from paper_2407_05433_gb300 import autograd as ag
    from oracle.adjoint import implicit_gradients
    from oracle.exact import exact_kkt
    pbs, batch, xrefs, xref = _config5(torch, ag)
    try:
        params = ag.batch_params(batch)
        _loss(torch, ag, batch, xref, params).backward()
        got = {k: p.grad.cpu().numpy() for k, p in zip(ag.PARAM_KEYS, params)}
        for j in SAMPLED:
            pb = pbs[j]
            e = exact_kkt(pb)
            G = implicit_gradients(pb, 2.0 * (e["x"] - xrefs[j]), 2.0 * e["u"], sparse=True)
            sl = _slices(pbs, j)
            for k in FIELDS:
                ref = np.asarray(G[k]).ravel()
                if ref.size == 0:
                    continue
                err = np.max(np.abs(got[k][sl[k]] - ref)) / max(1.0, np.max(np.abs(ref)))
                assert err <= 1e-9, (j, k, err)
    finally:
        batch.close()


def test_config5_full_batch_against_finite_differences_of_the_oracle():
    """Central differences (h = 1e-6) of the oracle's loss on the same three problems, one sampled entry
    per field; Q and R are stepped along symmetric directions.  With |l| about 1e4 per problem the
    difference quotient carries rounding of about eps |l| / h = 2e-6, so the bar is 2e-5 relative to
    max(1, |g|)."""
    import torch
    from paper_2407_05433_gb300 import autograd as ag
    pbs, batch, xrefs, xref = _config5(torch, ag)
    try:
        params = ag.batch_params(batch)
        _loss(torch, ag, batch, xref, params).backward()
        got = {k: p.grad.cpu().numpy() for k, p in zip(ag.PARAM_KEYS, params)}
    finally:
        batch.close()
    h = 1e-6
    rng = np.random.default_rng(9)

    def loss_j(pb, xr):
        s = oracle.solve(pb)
        assert s.ok
        return float(np.sum((s.x - xr) ** 2) + np.sum(s.u ** 2))

    for j in SAMPLED:
        pb, sl = pbs[j], _slices(pbs, j)
        for k in FIELDS:
            arr = np.asarray(getattr(pb, k), dtype=float)
            if arr.size == 0:
                continue
            idx = np.unravel_index(int(rng.integers(arr.size)), arr.shape)
            sym = k in ("Q", "R") and idx[-1] != idx[-2]

            def step(dh):
                q = pb.copy()
                a = np.array(getattr(q, k), dtype=float, copy=True)
                a[idx] += dh
                if sym:
                    a[tuple(idx[:-2]) + (idx[-1], idx[-2])] += dh
                setattr(q, k, a)
                return q

            fd = (loss_j(step(h), xrefs[j]) - loss_j(step(-h), xrefs[j])) / (2 * h)
            gj = got[k][sl[k]].reshape(arr.shape)
            g = gj[idx] + (gj[tuple(idx[:-2]) + (idx[-1], idx[-2])] if sym else 0.0)
            assert abs(fd - g) <= 2e-5 * max(1.0, abs(g)), (j, k, idx, fd, g)


def test_checkpointed_gradients_equal_the_stored_factor_gradients():
    """The checkpointed form (four segments of 256 problems on one segment-sized handle, factors
    recomputed in the backward pass) gives the gradients of the stored-factor form on the full
    differentiable batch, to 1e-10 (a segment of 256 problems takes the chunked schedule, the full
    batch one chunk per problem: the same arithmetic in another order)."""
    import torch
    from paper_2407_05433_gb300 import autograd as ag
    pbs, batch, xrefs, xref = _config5(torch, ag)
    seg = eclqr.Batch(pbs[:256])
    try:
        p1 = ag.batch_params(batch)
        _loss(torch, ag, batch, xref, p1).backward()
        p2 = [p.detach().clone().requires_grad_(True) for p in p1]
        x, u = ag.solve_checkpointed(seg, 4, *p2)
        (((x - xref) ** 2).sum() + (u ** 2).sum()).backward()
        for k, a, b in zip(ag.PARAM_KEYS, p1, p2):
            if a.numel() == 0:
                continue
            err = float((a.grad - b.grad).abs().max()) / max(1.0, float(a.grad.abs().max()))
            assert err <= 1e-10, (k, err)
    finally:
        seg.close()
        batch.close()
