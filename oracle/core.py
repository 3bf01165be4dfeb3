"""ctypes binding of the C oracle (``eclqr_oracle.c``).  Test infrastructure only.

The arrays handed in follow the packed layout of the problem statement
(Sec. 2, eq. problem): per-stage blocks, row-major, stage after stage.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "eclqr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

STATUS_NAMES = {0: "ok", 1: "infeasible_suffix", 2: "infeasible_x0", 3: "rank_inconsistent",
                4: "nonconvex", 6: "nonfinite", 7: "bad_input"}


def build_oracle(force=False, plant=0, out=None):
    """Compile the C oracle with plain IEEE double semantics (no FMA contraction).
    ``plant`` > 0 builds a mutant with one planted mistake (tests only) into ``out``."""
    target = out or _LIB
    if force or plant or not os.path.exists(target) or os.path.getmtime(target) < os.path.getmtime(_SRC):
        tmp = target + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared",
                               "-fPIC", f"-DORC_PLANT={int(plant)}", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, target)
    return target


class _Problem(ct.Structure):
    _fields_ = [("N", ct.c_int), ("n", ct.c_int), ("m", ct.c_int),
                ("p", ct.c_void_p), ("q", ct.c_void_p)] + \
               [(k, ct.c_void_p) for k in ("A", "B", "c", "C", "D", "d", "E", "e",
                                           "Q", "M", "R", "qv", "rv", "s0")]


class _Debug(ct.Structure):
    _fields_ = [(k, ct.c_void_p) for k in ("nbar", "mbar", "hrows", "H", "T", "t", "Y", "Z", "y",
                                           "Abar", "Bbar", "cbar", "Qbar", "Mbar", "Rbar", "qbar",
                                           "rbar", "kappa", "z", "v", "lrows", "L", "pi", "UT")]


class _Options(ct.Structure):
    _fields_ = [("tau_rank", ct.c_double), ("tau_inc", ct.c_double), ("refine", ct.c_int),
                ("kkt_refine", ct.c_int), ("refine_tol", ct.c_double)]


def _bind(path):
    lib = ct.CDLL(path)
    lib.orc_solve.restype = ct.c_int
    lib.orc_solve.argtypes = [ct.POINTER(_Problem), ct.POINTER(_Options)] + [ct.c_void_p] * 6 + \
        [ct.POINTER(ct.c_int), ct.POINTER(ct.c_double), ct.c_void_p]
    lib.orc_kkt_residual.restype = ct.c_double
    lib.orc_kkt_residual.argtypes = [ct.POINTER(_Problem)] + [ct.c_void_p] * 7
    lib.orc_phase_flops.restype = None
    lib.orc_phase_flops.argtypes = [ct.c_void_p]
    return lib


def load_mutant(plant, directory):
    """A separately built oracle with planted mistake ``plant`` (for pin-sensitivity tests)."""
    path = os.path.join(directory, f"liboracle_plant{int(plant)}.so")
    build_oracle(plant=plant, out=path)
    return _bind(path)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ct.CDLL(build_oracle())
            lib.orc_solve.restype = ct.c_int
            lib.orc_solve.argtypes = [ct.POINTER(_Problem), ct.POINTER(_Options)] + [ct.c_void_p] * 6 + \
                [ct.POINTER(ct.c_int), ct.POINTER(ct.c_double), ct.c_void_p]
            lib.orc_kkt_residual.restype = ct.c_double
            lib.orc_kkt_residual.argtypes = [ct.POINTER(_Problem)] + [ct.c_void_p] * 7
            lib.orc_project.restype = ct.c_int
            lib.orc_project.argtypes = [ct.c_void_p, ct.c_int, ct.c_int, ct.c_int, ct.c_void_p, ct.c_int,
                                        ct.c_double, ct.c_double, ct.c_void_p, ct.POINTER(ct.c_int),
                                        ct.c_void_p]
            lib.orc_tqr_solve.restype = ct.c_int
            lib.orc_tqr_solve.argtypes = [ct.c_void_p, ct.c_int, ct.c_int, ct.c_double, ct.c_void_p,
                                          ct.c_int, ct.c_void_p, ct.c_void_p, ct.POINTER(ct.c_double)]
            lib.orc_phase_flops.restype = None
            lib.orc_phase_flops.argtypes = [ct.c_void_p]
            _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data if a is not None and a.size else None


def _problem_struct(pb):
    keep = dict(p=np.ascontiguousarray(pb.p, dtype=np.int32), q=np.ascontiguousarray(pb.q, dtype=np.int32))
    for k in ("A", "B", "c", "C", "D", "d", "E", "e", "Q", "M", "R", "qv", "rv", "s0"):
        keep[k] = _f64(getattr(pb, k))
    s = _Problem(pb.N, pb.n, pb.m, _ptr(keep["p"]) or keep["p"].ctypes.data,
                 keep["q"].ctypes.data, *[keep[k].ctypes.data for k in
                                          ("A", "B", "c", "C", "D", "d", "E", "e", "Q", "M", "R",
                                           "qv", "rv", "s0")])
    return s, keep


@dataclass
class OracleSolution:
    status: int
    fail_stage: int
    x: np.ndarray
    u: np.ndarray
    lam: np.ndarray
    mu: np.ndarray
    eta: np.ndarray
    alpha: np.ndarray
    flops: float
    debug: dict | None = None
    phase_flops: np.ndarray | None = None

    @property
    def ok(self):
        return self.status == 0


def solve(pb, tau_rank=1e-10, tau_inc=1e-8, multipliers=True, debug=False, refine=2, kkt_refine=8,
          refine_tol=5e-10, lib=None):
    """Run O2 on one problem; returns an OracleSolution (numpy arrays).

    ``refine`` passes of refinement on the reduced LQR's residual run inside every solve;
    ``kkt_refine`` passes on the original KKT residual (Sec. 8 advice to check the original
    residuals, Sec. 5 linearity in the offsets) follow, each only while the Sec. 9 residual
    exceeds ``refine_tol``.  ``debug`` arrays describe the first (unrefined) solve."""
    lib = lib or _load()
    N, n, m = pb.N, pb.n, pb.m
    P, Qn = int(np.sum(pb.p)), int(np.sum(pb.q))
    s, keep = _problem_struct(pb)
    x = np.zeros((N + 1, n)); u = np.zeros((N, m))
    lam = np.zeros((N + 1, n)); mu = np.zeros(P); eta = np.zeros(Qn); alpha = np.zeros(n)
    fail = ct.c_int(-1); fl = ct.c_double(0.0)
    dbg_arrays = None
    dbgp = None
    if debug:
        dbg_arrays = dict(
            nbar=np.zeros(N + 1, np.int32), mbar=np.zeros(N, np.int32), hrows=np.zeros(N + 1, np.int32),
            H=np.zeros((N + 1, n, n + 1)), T=np.zeros((N + 1, n, n)), t=np.zeros((N + 1, n)),
            Y=np.zeros((N, m, n)), Z=np.zeros((N, m, m)), y=np.zeros((N, m)),
            Abar=np.zeros((N, n, n)), Bbar=np.zeros((N, n, m)), cbar=np.zeros((N, n)),
            Qbar=np.zeros((N + 1, n, n)), Mbar=np.zeros((N, n, m)), Rbar=np.zeros((N, m, m)),
            qbar=np.zeros((N + 1, n)), rbar=np.zeros((N, m)), kappa=np.zeros(N + 1),
            z=np.zeros((N + 1, n)), v=np.zeros((N, m)), lrows=np.zeros(N + 1, np.int32),
            L=np.zeros((N + 1, n, n + 1)), pi=np.zeros((N + 1, n)), UT=np.zeros((N + 1, n, n)))
        dbgp = ct.byref(_Debug(*[dbg_arrays[k].ctypes.data for k, _ in _Debug._fields_]))
    opt = _Options(tau_rank, tau_inc, refine, kkt_refine if multipliers else 0, refine_tol)
    st = lib.orc_solve(ct.byref(s), ct.byref(opt), x.ctypes.data, u.ctypes.data,
                       lam.ctypes.data if multipliers else None, _ptr(mu) or mu.ctypes.data,
                       _ptr(eta) or eta.ctypes.data, alpha.ctypes.data, ct.byref(fail), ct.byref(fl), dbgp)
    del keep
    ph = np.zeros(8)
    lib.orc_phase_flops(ph.ctypes.data)
    sol = OracleSolution(st, fail.value, x, u, lam, mu, eta, alpha, fl.value, dbg_arrays, ph[:7].copy())
    return sol


def kkt_residual(pb, x, u, lam, mu, eta, alpha, parts=False, lib=None):
    """Infinity-norm KKT residual of the original problem (Sec. 9 definition)."""
    lib = lib or _load()
    s, keep = _problem_struct(pb)
    arrs = [_f64(a) for a in (x, u, lam, mu, eta, alpha)]
    pr = np.zeros(4)
    r = lib.orc_kkt_residual(ct.byref(s), *[a.ctypes.data for a in arrs], pr.ctypes.data)
    del keep
    return (r, pr) if parts else r


def project_rows(M, groups, nkeep, tau_rank=1e-10, tau_inc=1e-8):
    """Lemma 1 on the rows of M = [groups... | kept | offset]; returns
    (group ranks, kept relation rows (k x (nkeep+1)), inconsistent flag)."""
    lib = _load()
    M = _f64(M).copy()
    r, nc = M.shape
    gs = np.ascontiguousarray(groups, dtype=np.int32)
    gr = np.zeros(max(1, len(groups)), np.int32)
    kr = ct.c_int(0)
    out = np.zeros((max(r, 1), nkeep + 1))
    inc = lib.orc_project(M.ctypes.data, r, nc, len(groups), gs.ctypes.data if len(groups) else None,
                          nkeep, tau_rank, tau_inc, gr.ctypes.data, ct.byref(kr), out.ctypes.data)
    return gr[:len(groups)], out[:kr.value].copy(), bool(inc)


def tqr_solve(K, b, tau_rank=1e-10):
    """Rank, orthonormal Q (last columns span null(K)), min-norm X with K X = -b,
    and the relative residual of the rows judged dependent."""
    lib = _load()
    K = _f64(K)
    b = _f64(b)
    if b.ndim == 1:
        b = b[:, None]
    rk, nk = K.shape
    X = np.zeros((nk, b.shape[1]))
    Q = np.zeros((nk, nk))
    res = ct.c_double(0.0)
    rank = lib.orc_tqr_solve(K.ctypes.data, rk, nk, tau_rank, b.ctypes.data, b.shape[1],
                             X.ctypes.data, Q.ctypes.data, ct.byref(res))
    return rank, Q, X, res.value
