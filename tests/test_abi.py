"""The C ABI library builds, loads and exports what include/eclqr.h declares
(no compute calls: these run without a GPU)."""
import ctypes as ct
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2407_05433_gb300 import build as build_mod
from paper_2407_05433_gb300 import eclqr, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "eclqr.h")


@pytest.fixture(scope="module")
def lib():
    build_mod.build()
    return eclqr.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(eclqr_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("eclqr_layout", "eclqr_create", "eclqr_build", "eclqr_solve", "eclqr_multipliers",
                     "eclqr_kkt_residual", "eclqr_destroy", "eclqr_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", eclqr.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (eclqr_[a-z_]+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    for f in declared_functions():
        assert hasattr(lib, f)


def test_strerror_and_defaults(lib):
    assert eclqr.eclqr_strerror(0) == "ok"
    assert "invalid" in eclqr.eclqr_strerror(-1)
    o = eclqr.eclqr_default_options()
    assert o.tau_rank == 1e-10 and o.tau_inc == 1e-8 and o.refine == 2 and o.chunk == 0 and o.team_warps == 0
    assert o.scan_skip == 1 and o.kkt_refine == 8 and o.refine_tol == 5e-10 and o.riccati_fp32 == 0
    assert o.persist == 0 and o.corr_refine == -1


def test_layout_sizes_match_packing(lib):
    pbs = [synth.config("single_n4", N=10), synth.config("batched_uneven", N=7, index=2),
           synth.config("table1", N=5)]
    h = eclqr.pack_host(pbs)
    rc, L = eclqr.eclqr_layout(eclqr.make_desc(h))
    assert rc == 0
    for k in eclqr.DATA_KEYS + ("s0",):
        assert getattr(L, k) == h[k].size, k
    assert L.x == sum((pb.N + 1) * pb.n for pb in pbs)
    assert L.u == sum(pb.N * pb.m for pb in pbs)
    assert L.mu == sum(int(pb.p.sum()) for pb in pbs) and L.eta == sum(int(pb.q.sum()) for pb in pbs)
    assert L.stages == sum(pb.N for pb in pbs)


@pytest.mark.parametrize("bad", ["N0", "n_too_big", "neg_rows", "no_problems"])
def test_invalid_descriptors_rejected_before_any_device_call(lib, bad):
    pb = synth.config("single_n4", N=6)
    h = eclqr.pack_host([pb])
    if bad == "N0":
        h["N"][0] = 0
    elif bad == "n_too_big":
        h["n"][0] = 1000
    elif bad == "neg_rows":
        h["p"][2] = -1
    d = eclqr.make_desc(h)
    if bad == "no_problems":
        d.num_problems = 0
    rc, _ = eclqr.eclqr_layout(d)
    assert rc == eclqr.EINVAL
    rc, hd = eclqr.eclqr_create(d, None)
    assert rc == eclqr.EINVAL and not hd.value


def test_invalid_scan_skip_option_rejected_before_any_device_call(lib):
    """eclqr_options.scan_skip is 0 or 1; anything else is rejected while the options are checked,
    before the handle touches the device."""
    o = eclqr.eclqr_default_options()
    o.scan_skip = 2
    rc, handle = eclqr.eclqr_create(eclqr.make_desc(_desc_arrays(8, 4, 2, 1, 0)), o)
    assert rc == eclqr.EINVAL and not handle


def test_null_handle_calls_are_rejected(lib):
    assert lib.eclqr_build(None, None, None, None) == eclqr.EINVAL
    assert lib.eclqr_solve(None, None, None, None, None, None) == eclqr.EINVAL
    assert lib.eclqr_scan_skipped(None, None, None) == eclqr.EINVAL
    assert eclqr.eclqr_launch_count(None) == 0
    lib.eclqr_destroy(None)


def _desc_arrays(N, n, m, p, q):
    h = {"N": np.array([N], np.int32), "n": np.array([n], np.int32), "m": np.array([m], np.int32),
         "p": np.full(N, p, np.int32), "q": np.zeros(N + 1, np.int32)}
    h["q"][N] = q
    return h


def test_dimensions_beyond_shared_memory_rejected_before_allocation(lib):
    """n = 32, m = 16 with 32 mixed rows and 32 terminal rows needs more shared memory per task
    than a CTA holds: eclqr_create says so (ECLQR_ESMEM) before any device allocation."""
    h = _desc_arrays(4, 32, 16, 32, 32)
    rc, handle = eclqr.eclqr_create(eclqr.make_desc(h))
    assert rc == eclqr.ESMEM and not handle
    assert "shared memory" in eclqr.eclqr_strerror(eclqr.ESMEM)


def test_autotuner_keeps_the_fastest_passing_trial():
    """The autotuners' selection rule: fastest among the trials that met the gate, else the smallest residual."""
    chunk_trials = [(0, 5.6, 7e-11, True), (6, 5.4, 8e-5, False), (8, 5.9, 1e-10, True)]
    assert eclqr._pick(chunk_trials)[0] == 0
    pair_trials = [(0, 1, 8.2, 1e-10, True), (0, 2, 6.3, 2e-11, True), (0, 4, 5.6, 2e-9, False)]
    assert eclqr._pick(pair_trials)[:2] == (0, 2)
    failing = [(0, 4, 5.6, 3e-9, False), (8, 4, 5.9, 2e-9, False)]
    assert eclqr._pick(failing)[:2] == (8, 4)
