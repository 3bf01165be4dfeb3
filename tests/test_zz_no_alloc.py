"""eclqr_kkt_residual_noalloc against eclqr_kkt_residual, through the C ABI.

The no-alloc entry point serves callers that cannot allocate device memory
when they need the residual check (real-time loops that forbid allocation
after start-up, or processes whose device memory is held by another
allocator).  It keeps its descriptors in a fixed device array shared by every
call, so the test calls it twice in a row -- the second call finds the first
call's contents in that array -- and compares both results with the handle
path's residual on the same inputs.  This file is named to be collected last.
"""
import ctypes as ct

import numpy as np
import pytest

from paper_2407_05433_gb300 import eclqr, synth


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2407_05433_gb300 import build as b
    b.build()
    eclqr.load()


def _noalloc(batch, sol=None):
    """Residual of the current (or given) solution through the no-alloc entry point."""
    import torch
    t = sol or {k: getattr(batch, k) for k in ("x", "u", "lam", "mu", "eta", "alpha")}
    out = torch.full((len(batch.problems),), -1.0, dtype=torch.float64, device=batch.device)
    rc = eclqr.eclqr_kkt_residual_noalloc(batch.desc, batch.data, batch.d["s0"].data_ptr(), t["x"].data_ptr(),
                                          t["u"].data_ptr(), t["lam"].data_ptr(), t["mu"].data_ptr(),
                                          t["eta"].data_ptr(), t["alpha"].data_ptr(), out.data_ptr(),
                                          batch._stream())
    assert rc == eclqr.OK, eclqr.eclqr_strerror(rc)
    torch.cuda.synchronize(batch.device)
    return out.cpu().numpy()


def _handle(batch, sol=None):
    import torch
    t = sol or {k: getattr(batch, k) for k in ("x", "u", "lam", "mu", "eta", "alpha")}
    out = torch.full((len(batch.problems),), -1.0, dtype=torch.float64, device=batch.device)
    rc = eclqr.eclqr_kkt_residual(batch.h, batch.d["s0"].data_ptr(), t["x"].data_ptr(), t["u"].data_ptr(),
                                  t["lam"].data_ptr(), t["mu"].data_ptr(), t["eta"].data_ptr(),
                                  t["alpha"].data_ptr(), out.data_ptr(), batch._stream())
    assert rc == eclqr.OK
    torch.cuda.synchronize(batch.device)
    return out.cpu().numpy()


def _close(a, b):
    # the same maxima of the same per-row values: equal up to the last bit in
    # practice; the tolerance of the parity tests (1e-9 relative) bounds it
    return np.all(np.abs(a - b) <= 1e-9 * np.maximum(1.0, np.abs(b)))


@pytest.mark.gpu
def test_noalloc_matches_handle_residual_twice():
    import torch
    pbs = [synth.config("single_n4", N=40), synth.config("batched_uneven", index=1, N=33),
           synth.config("table1", N=20), synth.config("batched_uneven", index=2, N=17)]
    batch = eclqr.Batch(pbs)
    try:
        batch.run()
        ref = _handle(batch)
        assert np.all(ref >= 0) and np.all(ref <= 1e-9)
        first = _noalloc(batch)
        second = _noalloc(batch)
        assert _close(first, ref), (first, ref)
        assert _close(second, ref), (second, ref)
        # a perturbed point: both paths see the same nonzero residual, twice
        pert = {k: getattr(batch, k).clone() for k in ("x", "u", "lam", "mu", "eta", "alpha")}
        pert["lam"] += 1e-3
        pert["x"][5] += 2e-3
        ref2 = _handle(batch, pert)
        assert np.all(ref2 > 1e-4)
        a, b = _noalloc(batch, pert), _noalloc(batch, pert)
        assert _close(a, ref2) and _close(b, ref2), (a, b, ref2)
    finally:
        batch.close()


def _desc(Ns, n=1, m=1):
    """Host descriptor arrays of problems with no constraint rows."""
    h = {"N": np.asarray(Ns, np.int32), "n": np.full(len(Ns), n, np.int32), "m": np.full(len(Ns), m, np.int32),
         "p": np.zeros(int(np.sum(Ns)), np.int32), "q": np.zeros(int(np.sum(Ns)) + len(Ns), np.int32)}
    return h, eclqr.make_desc(h)


def test_noalloc_rejects_batches_beyond_its_array():
    # the size check comes before any CUDA call: this runs without a GPU
    fake = 1 << 20            # never dereferenced
    data = eclqr.eclqr_data(*([fake] * len(eclqr.DATA_KEYS)))
    args = [fake] * 8
    h1, d1 = _desc([140000])         # 140001 stage records
    assert eclqr.eclqr_kkt_residual_noalloc(d1, data, *args, None) == eclqr.ETOOBIG
    h2, d2 = _desc([1] * 5000)                         # 5000 problems
    assert eclqr.eclqr_kkt_residual_noalloc(d2, data, *args, None) == eclqr.ETOOBIG
    assert "exceeds" in eclqr.eclqr_strerror(eclqr.ETOOBIG)
    h3, d3 = _desc([4])
    d3.num_problems = 0                                # invalid descriptors still read as EINVAL
    assert eclqr.eclqr_kkt_residual_noalloc(d3, data, *args, None) == eclqr.EINVAL


@pytest.mark.gpu
def test_noalloc_on_a_larger_then_a_smaller_different_batch():
    """Each call rewrites the shared array for its own batch: a call on a larger batch, then on a
    smaller batch of other shapes, each against the handle path on the same inputs."""
    big = [synth.config("batched_uneven", index=j, N=30 + j) for j in range(6)] + [synth.config("table1", N=25)]
    small = [synth.config("single_n4", N=9), synth.config("degenerate_n12", N=11)]
    out = []
    for pbs in (big, small):
        batch = eclqr.Batch(pbs)
        try:
            batch.run()
            ref = _handle(batch)
            got = _noalloc(batch)
            assert _close(got, ref), (got, ref)
            out.append(got)
        finally:
            batch.close()
    assert len(out[0]) == 7 and len(out[1]) == 2


@pytest.mark.gpu
def test_noalloc_refuses_a_capturing_stream():
    """The descriptors are copied from a host array that the next call rewrites, so a graph would
    replay stale descriptors: on a capturing stream the call returns ECLQR_ESTATE and enqueues nothing."""
    import torch
    batch = eclqr.Batch([synth.config("single_n4", N=9)])
    try:
        batch.run()
        _noalloc(batch)
        out = torch.zeros(1, dtype=torch.float64, device=batch.device)
        g = torch.cuda.CUDAGraph()
        rcs = []
        with torch.cuda.graph(g, capture_error_mode="relaxed"):
            rcs.append(eclqr.eclqr_kkt_residual_noalloc(
                batch.desc, batch.data, batch.d["s0"].data_ptr(), batch.x.data_ptr(), batch.u.data_ptr(),
                batch.lam.data_ptr(), batch.mu.data_ptr(), batch.eta.data_ptr(), batch.alpha.data_ptr(),
                out.data_ptr(), batch._stream()))
        assert rcs == [eclqr.ESTATE]
    finally:
        batch.close()
