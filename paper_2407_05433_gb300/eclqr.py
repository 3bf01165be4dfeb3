"""Thin Python binding of libeclqr.so, the C ABI declared in include/eclqr.h.

The functions named like the ABI (eclqr_layout, eclqr_create, eclqr_build,
eclqr_solve, eclqr_multipliers, eclqr_kkt_residual, ...) only marshal
arguments: every step of the reduction runs in the library's CUDA kernels.
``Batch`` packs a list of problems (see ``synth.ECLQRProblem`` for the packed
layout) into device tensors owned by torch and calls the ABI on torch's
current stream.  There is no CPU fallback: importing the binding without the
built library raises.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libeclqr.so")

OK, EINVAL, ENOMEM, ECUDA, ESTATE, ETOOBIG, ESMEM = 0, -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "ok", 1: "infeasible_suffix", 2: "infeasible_x0", 3: "rank_inconsistent",
                4: "nonconvex", 6: "nonfinite"}


class eclqr_desc(ct.Structure):
    _fields_ = [("num_problems", ct.c_int32), ("N", ct.c_void_p), ("n", ct.c_void_p), ("m", ct.c_void_p),
                ("p", ct.c_void_p), ("q", ct.c_void_p)]


class eclqr_data(ct.Structure):
    _fields_ = [(k, ct.c_void_p) for k in ("A", "B", "c", "C", "D", "d", "E", "e", "Q", "M", "R", "qv", "rv")]


class eclqr_grads(ct.Structure):
    _fields_ = [(k, ct.c_void_p) for k in ("A", "B", "c", "C", "D", "d", "E", "e", "Q", "M", "R", "qv", "rv", "s0")]


class eclqr_options(ct.Structure):
    _fields_ = [("tau_rank", ct.c_double), ("tau_inc", ct.c_double), ("refine", ct.c_int32), ("chunk", ct.c_int32),
                ("team_warps", ct.c_int32), ("scan_skip", ct.c_int32), ("kkt_refine", ct.c_int32),
                ("refine_tol", ct.c_double), ("riccati_fp32", ct.c_int32), ("persist", ct.c_int32),
                ("corr_refine", ct.c_int32)]


LAYOUT_FIELDS = ("A", "B", "c", "C", "D", "d", "E", "e", "Q", "M", "R", "qv", "rv", "s0",
                 "x", "u", "lam", "mu", "eta", "alpha", "stages")


class eclqr_layout_info(ct.Structure):
    _fields_ = [(k, ct.c_int64) for k in LAYOUT_FIELDS]


_lib = None


def load():
    """Load libeclqr.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libeclqr.so is not built ({LIB_PATH}); run paper_2407_05433_gb300/build.py")
    lib = ct.CDLL(LIB_PATH)
    vp, i32 = ct.c_void_p, ct.c_int
    lib.eclqr_default_options.argtypes = [ct.POINTER(eclqr_options)]
    lib.eclqr_default_options.restype = None
    lib.eclqr_layout.argtypes = [ct.POINTER(eclqr_desc), ct.POINTER(eclqr_layout_info)]
    lib.eclqr_layout.restype = i32
    lib.eclqr_create.argtypes = [ct.POINTER(eclqr_desc), ct.POINTER(eclqr_options), ct.POINTER(vp)]
    lib.eclqr_create.restype = i32
    lib.eclqr_build.argtypes = [vp, ct.POINTER(eclqr_data), vp, vp]
    lib.eclqr_build.restype = i32
    lib.eclqr_solve.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.eclqr_solve.restype = i32
    lib.eclqr_multipliers.argtypes = [vp] * 9
    lib.eclqr_multipliers.restype = i32
    lib.eclqr_kkt_residual.argtypes = [vp] * 10
    lib.eclqr_kkt_residual.restype = i32
    lib.eclqr_kkt_residual_parts.argtypes = [vp] * 11
    lib.eclqr_kkt_residual_parts.restype = i32
    lib.eclqr_refine.argtypes = [vp] * 11
    lib.eclqr_refine.restype = i32
    lib.eclqr_riccati_fp64_flags.argtypes = [vp, vp, vp]
    lib.eclqr_riccati_fp64_flags.restype = i32
    lib.eclqr_reduced_dims.argtypes = [vp, vp, vp, vp]
    lib.eclqr_reduced_dims.restype = i32
    lib.eclqr_scan_skipped.argtypes = [vp, vp, vp]
    lib.eclqr_scan_skipped.restype = i32
    lib.eclqr_launch_count.argtypes = [vp]
    lib.eclqr_launch_count.restype = ct.c_int64
    lib.eclqr_time_kernel.argtypes = [vp, ct.c_char_p]
    lib.eclqr_time_kernel.restype = i32
    lib.eclqr_kernel_time.argtypes = [vp, ct.POINTER(ct.c_int64), ct.POINTER(ct.c_double)]
    lib.eclqr_kernel_time.restype = i32
    lib.eclqr_probe_fp64_peak.argtypes = [ct.POINTER(ct.c_double)]
    lib.eclqr_probe_fp64_peak.restype = i32
    lib.eclqr_kkt_residual_noalloc.argtypes = [ct.POINTER(eclqr_desc), ct.POINTER(eclqr_data)] + [vp] * 9
    lib.eclqr_kkt_residual_noalloc.restype = i32
    lib.eclqr_param_grads.argtypes = [vp] * 13 + [ct.POINTER(eclqr_grads), vp]
    lib.eclqr_set_costs.argtypes = [vp, ct.POINTER(eclqr_data), vp]
    lib.eclqr_set_costs.restype = i32
    lib.eclqr_param_grads.restype = i32
    lib.eclqr_destroy.argtypes = [vp]
    lib.eclqr_destroy.restype = None
    lib.eclqr_strerror.argtypes = [i32]
    lib.eclqr_strerror.restype = ct.c_char_p
    _lib = lib
    return lib


def _check(rc, what):
    if rc != OK:
        raise RuntimeError(f"{what} failed: {load().eclqr_strerror(rc).decode()} ({rc})")


# ---------------------------------------------------------------- ABI-named calls (marshalling only)
def eclqr_default_options():
    o = eclqr_options()
    load().eclqr_default_options(ct.byref(o))
    return o


def eclqr_layout(desc):
    out = eclqr_layout_info()
    rc = load().eclqr_layout(ct.byref(desc), ct.byref(out))
    return rc, out


def eclqr_create(desc, opt=None):
    h = ct.c_void_p()
    rc = load().eclqr_create(ct.byref(desc), ct.byref(opt) if opt is not None else None, ct.byref(h))
    return rc, h


def eclqr_build(h, data, status, stream):
    return load().eclqr_build(h, ct.byref(data), status, stream)


def eclqr_solve(h, s0, x, u, status, stream):
    return load().eclqr_solve(h, s0, x, u, status, stream)


def eclqr_multipliers(h, x, u, lam, mu, eta, alpha, status, stream):
    return load().eclqr_multipliers(h, x, u, lam, mu, eta, alpha, status, stream)


def eclqr_kkt_residual(h, s0, x, u, lam, mu, eta, alpha, resid, stream):
    return load().eclqr_kkt_residual(h, s0, x, u, lam, mu, eta, alpha, resid, stream)


def eclqr_kkt_residual_parts(h, s0, x, u, lam, mu, eta, alpha, resid, parts, stream):
    return load().eclqr_kkt_residual_parts(h, s0, x, u, lam, mu, eta, alpha, resid, parts, stream)


def eclqr_refine(h, s0, x, u, lam, mu, eta, alpha, resid, status, stream):
    return load().eclqr_refine(h, s0, x, u, lam, mu, eta, alpha, resid, status, stream)


def eclqr_kkt_residual_noalloc(desc, data, s0, x, u, lam, mu, eta, alpha, resid, stream):
    return load().eclqr_kkt_residual_noalloc(ct.byref(desc), ct.byref(data), s0, x, u, lam, mu, eta, alpha,
                                             resid, stream)


def eclqr_param_grads(h, x, u, lam, mu, eta, alpha, xb, ub, lamb, mub, etab, alphab, out, stream):
    return load().eclqr_param_grads(h, x, u, lam, mu, eta, alpha, xb, ub, lamb, mub, etab, alphab,
                                    ct.byref(out), stream)


def eclqr_set_costs(h, data, stream):
    return load().eclqr_set_costs(h, ct.byref(data), stream)


def eclqr_reduced_dims(h, nbar, mbar, stream):
    return load().eclqr_reduced_dims(h, nbar, mbar, stream)


def eclqr_scan_skipped(h, flags, stream):
    return load().eclqr_scan_skipped(h, flags, stream)


def eclqr_launch_count(h):
    return int(load().eclqr_launch_count(h))


def eclqr_destroy(h):
    load().eclqr_destroy(h)


def eclqr_time_kernel(h, name):
    return load().eclqr_time_kernel(h, name.encode() if name else None)


def eclqr_kernel_time(h):
    n, t = ct.c_int64(0), ct.c_double(0.0)
    rc = load().eclqr_kernel_time(h, ct.byref(n), ct.byref(t))
    _check(rc, "eclqr_kernel_time")
    return int(n.value), float(t.value)


def eclqr_probe_fp64_peak():
    t = ct.c_double(0.0)
    _check(load().eclqr_probe_fp64_peak(ct.byref(t)), "eclqr_probe_fp64_peak")
    return float(t.value)


def eclqr_strerror(code):
    return load().eclqr_strerror(code).decode()


# ---------------------------------------------------------------- packing helpers
DATA_KEYS = ("A", "B", "c", "C", "D", "d", "E", "e", "Q", "M", "R", "qv", "rv")


def pack_host(problems):
    """Concatenate the packed arrays of several problems (problem after problem)."""
    out = {}
    for k in DATA_KEYS + ("s0",):
        out[k] = np.ascontiguousarray(np.concatenate([np.asarray(getattr(pb, k), np.float64).ravel()
                                                      for pb in problems]))
    out["N"] = np.array([pb.N for pb in problems], np.int32)
    out["n"] = np.array([pb.n for pb in problems], np.int32)
    out["m"] = np.array([pb.m for pb in problems], np.int32)
    out["p"] = np.ascontiguousarray(np.concatenate([np.asarray(pb.p, np.int32) for pb in problems]))
    out["q"] = np.ascontiguousarray(np.concatenate([np.asarray(pb.q, np.int32) for pb in problems]))
    return out


def make_desc(h):
    d = eclqr_desc()
    d.num_problems = len(h["N"])
    d.N, d.n, d.m = h["N"].ctypes.data, h["n"].ctypes.data, h["m"].ctypes.data
    d.p, d.q = h["p"].ctypes.data, h["q"].ctypes.data
    return d


class Batch:
    """A batch of problems resident on one CUDA device, solved through the C ABI."""

    def __init__(self, problems, device="cuda", tau_rank=1e-10, tau_inc=1e-8, refine=2, chunk=0, team_warps=0,
                 scan_skip=1, kkt_refine=8, refine_tol=5e-10, riccati_fp32=0, persist=0, corr_refine=-1):
        import torch
        self.torch = torch
        self.problems = list(problems)
        self.device = torch.device(device)
        self.host = pack_host(self.problems)
        self.desc = make_desc(self.host)
        rc, self.layout = eclqr_layout(self.desc)
        _check(rc, "eclqr_layout")
        opt = eclqr_default_options()
        opt.tau_rank, opt.tau_inc, opt.refine, opt.chunk = tau_rank, tau_inc, refine, chunk
        opt.team_warps = team_warps
        opt.scan_skip = scan_skip
        opt.kkt_refine, opt.refine_tol = kkt_refine, refine_tol
        opt.riccati_fp32 = riccati_fp32
        opt.persist = persist
        opt.corr_refine = corr_refine
        with torch.cuda.device(self.device):
            rc, self.h = eclqr_create(self.desc, opt)
        _check(rc, "eclqr_create")
        f64 = dict(dtype=torch.float64, device=self.device)
        self.d = {k: torch.from_numpy(self.host[k]).to(self.device) for k in DATA_KEYS + ("s0",)}
        L = self.layout
        self.x = torch.zeros(max(1, L.x), **f64)
        self.u = torch.zeros(max(1, L.u), **f64)
        self.lam = torch.zeros(max(1, L.lam), **f64)
        self.mu = torch.zeros(max(1, L.mu), **f64)
        self.eta = torch.zeros(max(1, L.eta), **f64)
        self.alpha = torch.zeros(max(1, L.alpha), **f64)
        self.resid = torch.zeros(len(self.problems), **f64)
        self.status = torch.zeros(len(self.problems), dtype=torch.int32, device=self.device)
        self.data = eclqr_data(*[self.d[k].data_ptr() for k in DATA_KEYS])

    def _stream(self):
        return ct.c_void_p(self.torch.cuda.current_stream(self.device).cuda_stream)

    def invalidate(self):
        """Marks the handle as holding another build than this Batch's own data (autograd builds on
        copies of the data): solve, multipliers, refine and residual then raise until build()."""
        self._own_build = False

    def _require_own_build(self, what):
        if not getattr(self, "_own_build", False):
            raise RuntimeError(f"{what}: the handle does not hold a build of this Batch's data; call build() first")

    def build(self):
        _check(eclqr_build(self.h, self.data, self.status.data_ptr(), self._stream()), "eclqr_build")
        self._own_build = True

    def solve(self, s0=None):
        self._require_own_build("solve")
        s0 = self.d["s0"] if s0 is None else s0
        _check(eclqr_solve(self.h, s0.data_ptr(), self.x.data_ptr(), self.u.data_ptr(), self.status.data_ptr(),
                           self._stream()), "eclqr_solve")

    def multipliers(self):
        self._require_own_build("multipliers")
        _check(eclqr_multipliers(self.h, self.x.data_ptr(), self.u.data_ptr(), self.lam.data_ptr(),
                                 self.mu.data_ptr(), self.eta.data_ptr(), self.alpha.data_ptr(),
                                 self.status.data_ptr(), self._stream()), "eclqr_multipliers")

    def residual(self, s0=None):
        self._require_own_build("residual")
        s0 = self.d["s0"] if s0 is None else s0
        _check(eclqr_kkt_residual(self.h, s0.data_ptr(), self.x.data_ptr(), self.u.data_ptr(),
                                  self.lam.data_ptr(), self.mu.data_ptr(), self.eta.data_ptr(),
                                  self.alpha.data_ptr(), self.resid.data_ptr(), self._stream()),
               "eclqr_kkt_residual")

    def residual_parts(self, s0=None):
        """Per problem the four parts of the Sec. 9 residual (initial condition, dynamics, normalised
        equality rows, stationarity) as a numpy (P, 4) array; also refreshes self.resid."""
        self._require_own_build("residual_parts")
        s0 = self.d["s0"] if s0 is None else s0
        parts = self.torch.zeros(4 * len(self.problems), dtype=self.torch.float64, device=self.device)
        _check(eclqr_kkt_residual_parts(self.h, s0.data_ptr(), self.x.data_ptr(), self.u.data_ptr(),
                                        self.lam.data_ptr(), self.mu.data_ptr(), self.eta.data_ptr(),
                                        self.alpha.data_ptr(), self.resid.data_ptr(), parts.data_ptr(),
                                        self._stream()), "eclqr_kkt_residual_parts")
        return parts.cpu().numpy().reshape(-1, 4)

    def refine(self, s0=None):
        """Refinement on the original KKT residual (eclqr_refine); leaves the residual in self.resid."""
        self._require_own_build("refine")
        s0 = self.d["s0"] if s0 is None else s0
        _check(eclqr_refine(self.h, s0.data_ptr(), self.x.data_ptr(), self.u.data_ptr(), self.lam.data_ptr(),
                            self.mu.data_ptr(), self.eta.data_ptr(), self.alpha.data_ptr(), self.resid.data_ptr(),
                            self.status.data_ptr(), self._stream()), "eclqr_refine")

    def run(self, multipliers=True, residual=True):
        """One pass of the path: build, solve and, with multipliers, the multipliers and the refinement
        on the original KKT residual, which leaves the Sec. 9 residual in self.resid."""
        self.build()
        self.solve()
        if multipliers:
            self.multipliers()
        if residual and multipliers:
            self.refine()

    def capture(self):
        """Capture one full pass (build, solve, multipliers, residual) into a CUDA graph.

        The graph keeps the current device pointers: refresh the inputs in place (self.d)
        and call replay().  A first eager pass on a side stream sets every kernel's
        shared-memory attribute before capture.  Returns the number of kernel launches
        one replay performs."""
        torch = self.torch
        side = torch.cuda.Stream(self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(side):
            self.run()
        torch.cuda.current_stream(self.device).wait_stream(side)
        torch.cuda.synchronize(self.device)
        before = self.launches()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, capture_error_mode="relaxed"):
            self.run()
        self.graph = graph
        self.graph_launches = self.launches() - before
        return self.graph_launches

    def replay(self):
        self.graph.replay()

    def riccati_fp64(self):
        """Per problem: True where the Riccati sweep ran in FP64 (always in FP64 mode; in mixed precision,
        the problems eclqr_refine redid in FP64)."""
        torch = self.torch
        f = torch.zeros(len(self.problems), dtype=torch.int32, device=self.device)
        _check(load().eclqr_riccati_fp64_flags(self.h, f.data_ptr(), self._stream()), "eclqr_riccati_fp64_flags")
        return f.cpu().numpy().astype(bool)

    def scan_skipped(self):
        """Per problem: True where the build skipped the feasible-domain scan (Sec. 6 shortcut)."""
        torch = self.torch
        f = torch.zeros(len(self.problems), dtype=torch.int32, device=self.device)
        _check(eclqr_scan_skipped(self.h, f.data_ptr(), self._stream()), "eclqr_scan_skipped")
        return f.cpu().numpy().astype(bool)

    def reduced_dims(self):
        torch = self.torch
        nb = torch.zeros(int(self.layout.x // 1), dtype=torch.int32, device=self.device)
        mb = torch.zeros(int(self.layout.u // 1), dtype=torch.int32, device=self.device)
        _check(eclqr_reduced_dims(self.h, nb.data_ptr(), mb.data_ptr(), self._stream()), "eclqr_reduced_dims")
        nb, mb = nb.cpu().numpy(), mb.cpu().numpy()
        out, ob, om = [], 0, 0
        for pb in self.problems:
            out.append((nb[ob:ob + pb.N + 1].copy(), mb[om:om + pb.N].copy()))
            ob += pb.N + 1
            om += pb.N
        return out

    def launches(self):
        return eclqr_launch_count(self.h)

    def results(self):
        """Per-problem numpy views of the outputs (synchronises the stream)."""
        self.torch.cuda.synchronize(self.device)
        host = {k: getattr(self, k).cpu().numpy() for k in ("x", "u", "lam", "mu", "eta", "alpha", "resid", "status")}
        res, o = [], dict(x=0, u=0, lam=0, mu=0, eta=0, alpha=0)
        for j, pb in enumerate(self.problems):
            P, Qr = int(np.sum(pb.p)), int(np.sum(pb.q))
            sizes = dict(x=(pb.N + 1) * pb.n, u=pb.N * pb.m, lam=(pb.N + 1) * pb.n, mu=P, eta=Qr, alpha=pb.n)
            r = {}
            for k, sz in sizes.items():
                r[k] = host[k][o[k]:o[k] + sz].copy()
                o[k] += sz
            r["x"] = r["x"].reshape(pb.N + 1, pb.n)
            r["u"] = r["u"].reshape(pb.N, pb.m)
            r["lam"] = r["lam"].reshape(pb.N + 1, pb.n)
            r["resid"] = float(host["resid"][j])
            r["status"] = int(host["status"][j])
            res.append(r)
        return res

    def close(self):
        if getattr(self, "h", None):
            eclqr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _timed_pass(problems, device, refine, passes, gate, **kw):
    """(ms per full pass, max KKT residual, passed) of one schedule; the first pass is untimed."""
    import torch
    b = Batch(problems, device=device, refine=refine, **kw)
    try:
        b.run()
        torch.cuda.synchronize(b.device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(passes):
            b.run()
        e1.record()
        torch.cuda.synchronize(b.device)
        ms = e0.elapsed_time(e1) / passes
        res = float(b.resid.max())
        ok = bool(int(b.status.abs().max()) == 0 and res <= gate)
    finally:
        b.close()
    return ms, res, ok


def _pick(trials):
    """The fastest passing trial, else the one with the smallest residual."""
    passing = [t for t in trials if t[-1]]
    return min(passing, key=lambda t: t[-3]) if passing else min(trials, key=lambda t: t[-2])


def autotune_chunk(problems, device="cuda", candidates=(0, 6, 8, 12, 16, 32, -1), gate=1e-9, refine=2, passes=3,
                   **kw):
    """Chunk length for these problems: the fastest full pass (build, solve, multipliers, residual) among
    the candidates whose every problem ends with status 0 and a KKT residual <= gate.

    0 is the automatic choice of eclqr_create, -1 one chunk per problem (a single team sweeps every
    stage).  The chunk boundaries place the scan's composed relations next to the sweeps' own sets,
    and where they meet the multipliers inherit the difference, so which lengths pass depends on the
    instance.  Returns (chunk, trials) with trials = [(chunk, ms, max residual, passed)].  When no
    candidate passes, the one with the smallest residual is returned."""
    trials = []
    for L in candidates:
        chunk = max(pb.N for pb in problems) if L == -1 else L
        trials.append((chunk,) + _timed_pass(problems, device, refine, passes, gate, chunk=chunk, **kw))
    return _pick(trials)[0], trials


def autotune_schedule(problems, device="cuda", chunks=(0, 8, 16, -1), teams=(1, 2, 4), gate=1e-9, refine=2,
                      passes=3, **kw):
    """Schedule for these problems: chunk length (as in autotune_chunk) and team size, the warps of the
    CTA that composes one relation (1 = a warp per relation, 4 = the default CTA).  Small relations
    (n of a few states) leave most of a four-warp team idle; large ones need it.  Every pair is timed
    over full passes and gated like autotune_chunk.  Returns ((chunk, team_warps), trials) with
    trials = [(chunk, team_warps, ms, max residual, passed)]."""
    trials = []
    for L in chunks:
        chunk = max(pb.N for pb in problems) if L == -1 else L
        for w in teams:
            trials.append((chunk, w) + _timed_pass(problems, device, refine, passes, gate, chunk=chunk,
                                                   team_warps=w, **kw))
    best = _pick(trials)
    return (best[0], best[1]), trials
