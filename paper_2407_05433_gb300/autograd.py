"""Differentiable solve: x, u of a batch as functions of its packed data.

Backward is implicit differentiation of the KKT system through the C ABI
(eclqr_param_grads): the adjoint is the solution of the same problems with
the same matrices, the incoming gradients as linear costs (q' = -dl/dx,
r' = -dl/du) and zero c, d, e, s0.  When the handle still holds the factors
of this forward pass, the adjoint reuses them (eclqr_set_costs, then
eclqr_solve and eclqr_multipliers: no new build); otherwise the factors are
rebuilt on the adjoint data.  The gradients are outer products of solution
and adjoint, one CTA per stage.  Gradients of Q_i and R_i are symmetrised.
"""
from __future__ import annotations

import torch

from . import eclqr

PARAM_KEYS = eclqr.DATA_KEYS + ("s0",)
_OFFSETS = ("c", "d", "e")


def batch_params(batch, requires_grad=True):
    """Copies of a Batch's packed device data, one tensor per key of PARAM_KEYS."""
    return [batch.d[k].detach().clone().requires_grad_(requires_grad) for k in PARAM_KEYS]


def _run(batch, data_tensors, s0, reuse=False):
    """build (or, with reuse, eclqr_set_costs on the last build's factors) + solve + multipliers +
    refinement on the original KKT residual, on the given data; returns the six packed outputs and
    status.  The handle then points at data_tensors, not at batch.data: the Batch is marked so that
    its own solve, multipliers and residual calls refuse to run until its next build()."""
    L = batch.layout
    f64 = dict(dtype=torch.float64, device=batch.device)
    out = [torch.zeros(max(1, int(getattr(L, k))), **f64) for k in ("x", "u", "lam", "mu", "eta", "alpha")]
    status = torch.zeros(len(batch.problems), dtype=torch.int32, device=batch.device)
    resid = torch.zeros(len(batch.problems), **f64)
    data = eclqr.eclqr_data(*[t.data_ptr() for t in data_tensors])
    st = batch._stream()
    batch.invalidate()
    if reuse:
        eclqr._check(eclqr.eclqr_set_costs(batch.h, data, st), "eclqr_set_costs")
    else:
        eclqr._check(eclqr.eclqr_build(batch.h, data, status.data_ptr(), st), "eclqr_build")
        batch._factor_token = getattr(batch, "_factor_token", 0) + 1
    eclqr._check(eclqr.eclqr_solve(batch.h, s0.data_ptr(), out[0].data_ptr(), out[1].data_ptr(), status.data_ptr(),
                                   st), "eclqr_solve")
    eclqr._check(eclqr.eclqr_multipliers(batch.h, *[t.data_ptr() for t in out], status.data_ptr(), st),
                 "eclqr_multipliers")
    eclqr._check(eclqr.eclqr_refine(batch.h, s0.data_ptr(), *[t.data_ptr() for t in out], resid.data_ptr(),
                                    status.data_ptr(), st), "eclqr_refine")
    return out, status


class ECLQRSolve(torch.autograd.Function):
    """forward(batch, *params) -> (x, u), params in PARAM_KEYS order (packed float64 on batch.device)."""

    reuse_factors = True  # backward reuses the forward build's factors when the handle still holds them

    @staticmethod
    def forward(ctx, batch, *params):
        params = [p.detach().contiguous() for p in params]
        out, status = _run(batch, params[:-1], params[-1])
        ctx.batch = batch
        ctx.token = batch._factor_token
        ctx.save_for_backward(*params, *out, status)
        L = batch.layout
        x, u = out[0][:int(L.x)], out[1][:int(L.u)]
        return x.clone(), u.clone()

    @staticmethod
    def backward(ctx, gx, gu):
        batch = ctx.batch
        saved = ctx.saved_tensors
        nk = len(PARAM_KEYS)
        params, sol, status = saved[:nk], saved[nk:nk + 6], saved[nk + 6]
        if int(status.abs().max()) != 0:
            raise RuntimeError("eclqr forward solve reported a nonzero status; no gradient")
        L = batch.layout
        f64 = dict(dtype=torch.float64, device=batch.device)
        lx = torch.zeros(max(1, int(L.x)), **f64)
        lu = torch.zeros(max(1, int(L.u)), **f64)
        if gx is not None:
            lx[:int(L.x)] = gx
        if gu is not None:
            lu[:int(L.u)] = gu
        adj = {k: p for k, p in zip(PARAM_KEYS, params)}
        for k in _OFFSETS:
            adj[k] = torch.zeros_like(adj[k])
        adj["qv"] = -lx[:adj["qv"].numel()]
        adj["rv"] = -lu[:adj["rv"].numel()]
        s0b = torch.zeros_like(adj["s0"])
        adjd = [adj[k].contiguous() for k in eclqr.DATA_KEYS]
        reuse = getattr(batch, "_factor_token", None) == ctx.token and ECLQRSolve.reuse_factors
        wb, st_b = _run(batch, adjd, s0b, reuse=reuse)
        grads = [torch.zeros_like(p) for p in params]
        g = eclqr.eclqr_grads(*[t.data_ptr() for t in grads])
        eclqr._check(eclqr.eclqr_param_grads(batch.h, *[t.data_ptr() for t in sol], *[t.data_ptr() for t in wb], g,
                                             batch._stream()), "eclqr_param_grads")
        if int(st_b.abs().max()) != 0:
            raise RuntimeError("eclqr adjoint solve reported a nonzero status")
        return (None, *grads)


def solve(batch, *params):
    """Differentiable x, u (packed) of batch's problems with the given data (PARAM_KEYS order)."""
    return ECLQRSolve.apply(batch, *params)


class ECLQRSolveCheckpointed(torch.autograd.Function):
    """Checkpointed form for a batch of S segments of identical structure: seg is a Batch of one
    segment (its problems' structure repeats S times in the packed params).  The forward pass solves
    the segments one after another on seg's handle and keeps only their solutions; the backward pass
    rebuilds each segment's factors from its data (the scan factors recomputed instead of stored)
    and runs the adjoint on them.  Device workspace: one segment's instead of the batch's, at the
    price of one more build per segment in the backward pass.

    forward(seg, S, *params) -> (x, u), params in PARAM_KEYS order for all S segments."""

    @staticmethod
    def forward(ctx, seg, S, *params):
        L = seg.layout
        sizes = {k: int(getattr(L, k)) for k in PARAM_KEYS}
        outs = {k: [] for k in ("x", "u", "lam", "mu", "eta", "alpha")}
        for j in range(S):
            sl = [p.detach()[j * sizes[k]:(j + 1) * sizes[k]].contiguous() for k, p in zip(PARAM_KEYS, params)]
            out, status = _run(seg, sl[:-1], sl[-1])
            if int(status.abs().max()) != 0:
                raise RuntimeError("eclqr forward solve reported a nonzero status")
            for k, t in zip(outs, out):
                outs[k].append(t[:int(getattr(L, k))].clone())
        sol = [torch.cat(outs[k]) for k in outs]
        ctx.seg, ctx.S = seg, S
        ctx.save_for_backward(*[p.detach() for p in params], *sol)
        return sol[0].clone(), sol[1].clone()

    @staticmethod
    def backward(ctx, gx, gu):
        seg, S = ctx.seg, ctx.S
        nk = len(PARAM_KEYS)
        saved = ctx.saved_tensors
        params, sol = saved[:nk], saved[nk:]
        L = seg.layout
        f64 = dict(dtype=torch.float64, device=seg.device)
        sizes = {k: int(getattr(L, k)) for k in PARAM_KEYS}
        osz = {k: int(getattr(L, k)) for k in ("x", "u", "lam", "mu", "eta", "alpha")}
        grads = [torch.zeros_like(p) for p in params]
        for j in range(S):
            sl = {k: p[j * sizes[k]:(j + 1) * sizes[k]].contiguous() for k, p in zip(PARAM_KEYS, params)}
            w = [torch.zeros(max(1, v), **f64) for v in osz.values()]
            for t, (k, v) in zip(w, osz.items()):
                t[:v] = sol[list(osz).index(k)][j * v:(j + 1) * v]
            # the forward factors of this segment, recomputed
            _run(seg, [sl[k] for k in eclqr.DATA_KEYS], sl["s0"])
            lx = torch.zeros(max(1, osz["x"]), **f64)
            lu = torch.zeros(max(1, osz["u"]), **f64)
            if gx is not None:
                lx[:osz["x"]] = gx[j * osz["x"]:(j + 1) * osz["x"]]
            if gu is not None:
                lu[:osz["u"]] = gu[j * osz["u"]:(j + 1) * osz["u"]]
            adj = dict(sl)
            for k in _OFFSETS:
                adj[k] = torch.zeros_like(adj[k])
            adj["qv"] = -lx[:sizes["qv"]]
            adj["rv"] = -lu[:sizes["rv"]]
            wb, st_b = _run(seg, [adj[k].contiguous() for k in eclqr.DATA_KEYS], torch.zeros_like(sl["s0"]),
                            reuse=True)
            if int(st_b.abs().max()) != 0:
                raise RuntimeError("eclqr adjoint solve reported a nonzero status")
            gj = [torch.zeros(max(1, sizes[k]), **f64) for k in PARAM_KEYS]
            g = eclqr.eclqr_grads(*[t.data_ptr() for t in gj])
            eclqr._check(eclqr.eclqr_param_grads(seg.h, *[t.data_ptr() for t in w], *[t.data_ptr() for t in wb], g,
                                                 seg._stream()), "eclqr_param_grads")
            for gr, t, k in zip(grads, gj, PARAM_KEYS):
                gr[j * sizes[k]:(j + 1) * sizes[k]] = t[:sizes[k]]
        return (None, None, *grads)


def solve_checkpointed(seg, segments, *params):
    """Differentiable x, u (packed) of `segments` copies of seg's structure with the given data
    (PARAM_KEYS order, all segments back to back); factors are recomputed in the backward pass."""
    return ECLQRSolveCheckpointed.apply(seg, segments, *params)
