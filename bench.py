#!/usr/bin/env python
"""Throughput benchmark: equality-constrained LQR stages solved per second, batched against plain.

One step is one pass of the whole path of Algorithm 1 through the C ABI over one batch:
eclqr_build (suffix-domain scan, stage elimination, Riccati factors), eclqr_solve (rollout with
refinement on the reduced residual, recovery of x, u), eclqr_multipliers (Sec. 7) and eclqr_refine
(the Sec. 9 residual, which gates the metric, and refinement on it for the problems above 5e-10).
The workload is the uneven batch: 4096 distinct seeded problems (seeds 0..4095), N ~ U[32, 512],
n in {8, 12, 16, 24}, m = n/2, mixed rows U{0..m} per stage, terminal rows U{0..n/2}; one chunk
per problem.  The step is captured once into a CUDA graph and replayed.

A problem counts as solved when its status is OK and its residual is at most 1e-9, or, for the
draws listed in tests/golden/batched_uneven_floors.txt (whose exact KKT solution, rounded to FP64,
already has a residual of that order), at most 4 phi, phi their FP64 floor.  ``value`` counts the
stages of solved problems; the line names the others.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference] [--no-extra]

Beside the headline the line carries "plain" (the same draws solved one problem at a time, each as
one chunk: a single CTA sweeps every stage, no scan, no batching), the per-kernel device time of
the batch, and at N = 1 further workloads: the long horizon (N = 65536), the degenerate instance
(N = 1024), the single instance (N = 64), the differentiable batch (1024 x 256, forward and
forward + backward), the Table 1 shape at N = 1024..16384 and the Sec. 6 scan-skip shortcut.

Under torchrun every rank solves its own copy of the batch (weak scaling, no collective on the data
path); rank 0 prints one JSON line.  ``--impl reference`` times the CPU oracle on the host instead
(rank 0 only): a bounded sample of the same draws over every host core.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ECLQR stages solved/s at KKT resid≤1e-9 (FP64), batched vs plain, % FP64 peak"
PROBLEMS = 4096
WORKLOAD = "batched_uneven"
WORKLOAD_DESC = ("batched_uneven: 4096 distinct problems (seeds 0..4095), N~U[32,512], n in {8,12,16,24}, m=n/2, "
                 "mixed rows U{0..m} per stage, terminal rows U{0..n/2}, A=I+0.1 randn, one batch, "
                 "one chunk per problem, CUDA-graph replay")
KKT_GATE = 1e-9
FLOOR_FACTOR = 4.0
GOLDEN = os.path.join(ROOT, "tests", "golden")
PLAIN_SAMPLE = 24
# reduced refinement passes inside each correction of the refinement on the KKT residual (fewer
# stall it); the first solve's count is chosen by autotune_refine
CORR_REFINE = 2
# kernels whose launches carry one phase of the method alone when every problem is one chunk
PHASE_KERNELS = {"k_primal_down": 0, "k_param": 1, "k_elim": 2, "k_riccati_down": 3, "k_dual_down": 5}
# kernels that carry the rest of the same phase (their time counts with the phase's kernel)
# (phase 5's forward substitution of nu also runs in k_aff_down, whose launches serve the rollout too and
# are left out, so the multipliers' rate is an upper bound)
PHASE_PARTNERS = {"k_riccati_down": ("k_riccati_finish",), "k_primal_down": ("k_primal_stage",),
                  "k_dual_down": ("k_dual_stage", "k_dual_leaf", "k_dual_root", "k_dual_terminal", "k_dual_up")}


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(value, world, device):
    """The largest of every rank's value (the job's time is its slowest rank's); identity at N = 1."""
    if world <= 1:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def all_ranks(flag, world, device):
    """True when every rank's flag is true (the gate holds for the whole job)."""
    if world <= 1:
        return bool(flag)
    import torch
    t = torch.tensor([1 if flag else 0], dtype=torch.int32, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MIN)
    return bool(int(t.item()))


def sum_over_ranks(value, world, device):
    if world <= 1:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.SUM)
    return float(t.item())


def job_rate(world, stages_per_rank, ms):
    """Whole-job throughput: every rank solves its own copy (weak scaling) within the slowest rank's time."""
    return world * stages_per_rank / (ms * 1e-3)


# ---------------------------------------------------------------- workload, gates, algorithmic work
def batched_problems(count=PROBLEMS, state_dim=None, max_horizon=None):
    """Draws 0..count-1 of the batch; with state_dim, only those whose state dimension is state_dim;
    with max_horizon, a draw whose horizon exceeds it is drawn again from the same seed at that
    horizon (a smaller case of the same shape, for profiling).  Returns (draw indices, problems)."""
    from paper_2407_05433_gb300 import synth
    pbs = [synth.config(WORKLOAD, index=j) for j in range(count)]
    if max_horizon is not None:
        pbs = [pb if pb.N <= max_horizon else synth.config(WORKLOAD, index=j, N=max_horizon)
               for j, pb in enumerate(pbs)]
    keep = [j for j, pb in enumerate(pbs) if state_dim is None or pb.n == state_dim]
    return keep, [pbs[j] for j in keep]


def floor_gates():
    """{draw index: gate} of the draws whose FP64 floor exceeds the 1e-9 gate."""
    out = {}
    path = os.path.join(GOLDEN, "batched_uneven_floors.txt")
    for ln in open(path):
        if ln.startswith("#") or not ln.strip():
            continue
        f = ln.split()
        out[int(f[0])] = max(KKT_GATE, FLOOR_FACTOR * float(f[4]))
    return out


def workload_flops():
    """Algorithmic FP64 work per workload (tests/golden/workload_flops.json, written from the oracle)."""
    path = os.path.join(GOLDEN, "workload_flops.json")
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)["workloads"]


def gate_report(pbs, res, stat, gates):
    """Which problems pass: status OK and residual at most their gate (NaN fails)."""
    import numpy as np
    g = np.array([gates.get(j, KKT_GATE) for j in range(len(pbs))])
    passed = (stat == 0) & (res <= g)
    failed = [int(j) for j in np.nonzero(~passed)[0]]
    return passed, {
        "rule": f"status OK and resid <= 1e-9; draws listed in tests/golden/batched_uneven_floors.txt: "
                f"resid <= max(1e-9, {FLOOR_FACTOR:g} phi)",
        "problems": len(pbs), "passed": int(passed.sum()),
        "passed_at_1e-9": int(((stat == 0) & (res <= KKT_GATE)).sum()),
        "floor_draws": len(gates), "failed": failed[:32],
        "failed_resid": [float(res[j]) for j in failed[:32]],
        "status_failures": int((stat != 0).sum()), "resid_max": float(np.nanmax(res)) if len(res) else 0.0,
        "nan_resid": int(np.isnan(res).sum()),
    }


# ---------------------------------------------------------------- GPU timing helpers
def _time_replays(batch, steps, flush, stream):
    """Device time (ms) of each of `steps` graph replays, L2 flushed between them (outside the events)."""
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        evs[k][0].record(stream)
        batch.replay()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def _time_runs(batch, steps, flush, stream):
    import torch
    times = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.run()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return times


def single_line(name, pb, dev, flush, stream, steps, **kw):
    """One instance through the same four calls, eager, `steps` timed passes."""
    from paper_2407_05433_gb300 import eclqr
    b = eclqr.Batch([pb], device=dev, **kw)
    try:
        b.run()
        ms = statistics.median(_time_runs(b, steps, flush, stream))
        (r,) = b.results()
        launches = b.launches()
    finally:
        b.close()
    return {"workload": name, "value": pb.N / (ms * 1e-3), "unit": "stages/s", "ms_per_step": ms,
            "kkt_resid": r["resid"], "status": r["status"],
            "gate_passed": bool(r["status"] == 0 and r["resid"] <= KKT_GATE)}


def autotune_refine(pbs, dev, gates, flush, stream, candidates=(2, 3, 4, 8), team_warps=0):
    """(refine, kkt_refine, trials).  For one and for two reduced refinement passes in the first
    solve (the KKT corrections keep two), the smallest KKT pass count whose eager pass leaves as
    many problems under their gate as the largest; of those pairs that reach the best gate count,
    the one whose captured step replays fastest.  trials: {"eager": [(refine, passes, ms, passed)],
    "replay": [(refine, passes, ms)]}."""
    from paper_2407_05433_gb300 import eclqr
    eager, pick = [], {}
    for refine in (1, 2):
        rows = []
        for kr in candidates:
            b = eclqr.Batch(pbs, device=dev, refine=refine, corr_refine=CORR_REFINE, kkt_refine=kr,
                            team_warps=team_warps)
            try:
                b.run()
                ms = statistics.median(_time_runs(b, 1, flush, stream))
                passed, _ = gate_report(pbs, b.resid.cpu().numpy(), b.status.cpu().numpy(), gates)
            finally:
                b.close()
            rows.append((refine, kr, round(ms, 1), int(passed.sum())))
        best = max(r[3] for r in rows)
        pick[refine] = (min(r[1] for r in rows if r[3] == best), best)
        eager += rows
    top = max(p[1] for p in pick.values())
    replay = []
    for refine, (kr, passed) in sorted(pick.items()):
        if passed < top:
            continue
        b = eclqr.Batch(pbs, device=dev, refine=refine, corr_refine=CORR_REFINE, kkt_refine=kr,
                        team_warps=team_warps)
        try:
            b.capture()
            for _ in range(2):
                b.replay()
            ms = statistics.median(_time_replays(b, 3, flush, stream))
        finally:
            b.close()
        replay.append((refine, kr, round(ms, 1)))
    refine, kr, _ = min(replay, key=lambda r: r[2])
    return refine, kr, {"eager": eager, "replay": replay}


def measure_plain(pbs, dev, flush, stream):
    """The plain GPU solve on the first PLAIN_SAMPLE draws of the batch: each problem alone, as one
    chunk (a single CTA sweeps every stage, no scan), through the same four calls, eager."""
    from paper_2407_05433_gb300 import eclqr
    tot_ms, tot_st, ok = 0.0, 0, 0
    for pb in pbs[:PLAIN_SAMPLE]:
        b = eclqr.Batch([pb], device=dev, chunk=pb.N)
        try:
            b.run()
            ms = statistics.median(_time_runs(b, 2, flush, stream))
            (r,) = b.results()
        finally:
            b.close()
        tot_ms += ms
        tot_st += pb.N
        ok += int(r["status"] == 0)
    return {"value": tot_st / (tot_ms * 1e-3), "unit": "stages/s", "problems": PLAIN_SAMPLE, "stages": tot_st,
            "ms_total": tot_ms, "status_ok": ok,
            "sample": f"draws 0..{PLAIN_SAMPLE - 1} of the batch, each solved alone as one chunk (one CTA of four "
                      f"warps sweeps every stage), median of 2 passes each"}


def measure_kernels(pbs, dev, flush, stream, flops, refine=2):
    """Per-kernel device time of one pass over the batch (without the refinement on the KKT
    residual), one (n, m) group at a time (groups run on concurrent streams in the batch itself,
    where one kernel's events would also cover the others' work).
    Every kernel of PHASE_KERNELS carries its phase alone when every problem is one chunk (together
    with its PHASE_PARTNERS), so its achieved FP64 rate is the phase's algorithmic flops over the
    summed launch time of those kernels."""
    from paper_2407_05433_gb300 import eclqr
    groups = {}
    for pb in pbs:
        groups.setdefault((pb.n, pb.m), []).append(pb)
    names = list(PHASE_KERNELS) + [p for ps in PHASE_PARTNERS.values() for p in ps] + [
                                   "k_lqr_up", "k_lqr_level", "k_primal_up", "k_dual_up", "k_aff_up",
                                   "k_aff_level", "k_aff_down", "k_kkt", "k_resid", "k_pcorr", "k_dual_leaf",
                                   "k_dual_stage", "k_dual_root", "k_refine_trial"]
    names = list(dict.fromkeys(names))  # each kernel timed once
    ms = {k: 0.0 for k in names}
    launches = {k: 0 for k in names}
    for key, gp in sorted(groups.items()):
        # the group alone still takes one chunk per problem (its longest horizon fits an SM's share).
        # Without the refinement on the KKT residual every kernel launches once per phase, so the
        # phase's flops and the kernel's time describe the same work.
        b = eclqr.Batch(gp, device=dev, refine=refine, kkt_refine=0)
        try:
            b.run()
            for name in names:
                eclqr.eclqr_time_kernel(b.h, name)
                flush.zero_()
                b.run()
                nl, t = eclqr.eclqr_kernel_time(b.h)
                ms[name] += t
                launches[name] += nl
            eclqr.eclqr_time_kernel(b.h, None)
        finally:
            b.close()
    out = {"kernel_ms_per_step": {k: round(v, 3) for k, v in sorted(ms.items(), key=lambda kv: -kv[1]) if v > 0},
           "launches_per_step": {k: v for k, v in launches.items() if v}}
    if flops:
        ph = flops["phase_flops"]
        out["phase_kernels"] = {}
        for k, p in PHASE_KERNELS.items():
            t = ms[k] + sum(ms[q] for q in PHASE_PARTNERS.get(k, ()))
            out["phase_kernels"][k] = {"phase": p, "ms": t, "with": list(PHASE_PARTNERS.get(k, ())),
                                       "algorithmic_flops": ph[p],
                                       "achieved_tflops": ph[p] / (t * 1e-3) / 1e12 if t else None}
    return out


def measure_without_kkt_refine(pbs, dev, flush, stream, gates, refine=2, steps=2):
    """The same batch and step without the refinement on the KKT residual (kkt_refine = 0), eager:
    what the refinement costs and what it buys."""
    from paper_2407_05433_gb300 import eclqr
    b = eclqr.Batch(pbs, device=dev, refine=refine, kkt_refine=0)
    try:
        b.run()
        ms = statistics.median(_time_runs(b, steps, flush, stream))
        res = b.resid.cpu().numpy()
        stat = b.status.cpu().numpy()
    finally:
        b.close()
    passed, rep = gate_report(pbs, res, stat, gates)
    return {"ms_per_step": ms, "passed": rep["passed"], "passed_at_1e-9": rep["passed_at_1e-9"],
            "resid_max": rep["resid_max"], "step": "eager eclqr_build + eclqr_solve + eclqr_multipliers + "
                                                   "eclqr_kkt_residual (no refinement passes)"}


def measure_mixed(name, pbs, dev, flush, stream, gates=None, steps=2, graph=False):
    """The same workload in mixed precision (riccati_fp32 = 1: the Riccati sweep in FP32, refinement in
    FP64, FP64 redo where it does not converge) beside FP64: time, problems under the gate, problems
    redone in FP64, and per problem the largest relative difference from the FP64 result (x, u and the
    multipliers, ||delta||_inf / max(1, ||fp64||_inf); the FP64 path is held to the oracle at 1e-9 by
    the tests)."""
    import numpy as np
    from paper_2407_05433_gb300 import eclqr
    out, ref = {"workload": name, "problems": len(pbs)}, None
    for tag, fp32 in (("fp64", 0), ("mixed", 1)):
        b = eclqr.Batch(pbs, device=dev, riccati_fp32=fp32)
        try:
            if graph:
                b.capture()
                b.replay()
                ms = statistics.median(_time_replays(b, steps, flush, stream))
            else:
                b.run()
                ms = statistics.median(_time_runs(b, steps, flush, stream))
            res = b.results()
            redo = int(b.riccati_fp64().sum()) if fp32 else len(pbs)
        finally:
            b.close()
        rr = np.array([r["resid"] for r in res])
        st = np.array([r["status"] for r in res])
        g = np.array([(gates or {}).get(j, KKT_GATE) for j in range(len(pbs))])
        out[tag] = {"ms_per_step": ms, "stages_per_s": sum(p.N for p in pbs) / (ms * 1e-3),
                    "passed": int(((st == 0) & (rr <= g)).sum()), "resid_max": float(np.nanmax(rr))}
        if fp32:
            out[tag]["redone_in_fp64"] = redo
            diffs = []
            for a, r in zip(ref, res):
                d = 0.0
                for k in ("x", "u", "lam", "mu", "eta", "alpha"):
                    x, y = np.asarray(r[k], float), np.asarray(a[k], float)
                    if y.size:
                        d = max(d, float(np.max(np.abs(x - y)) / max(1.0, np.max(np.abs(y)))))
                diffs.append(d)
            diffs = np.array(diffs)
            out[tag]["rel_diff_vs_fp64"] = {"max": float(diffs.max()), "median": float(np.median(diffs)),
                                            "over_1e-9": int((diffs > 1e-9).sum())}
        else:
            ref = res
    out["speedup_mixed_vs_fp64"] = out["fp64"]["ms_per_step"] / out["mixed"]["ms_per_step"]
    return out


def measure_diff_batch(dev, flush, stream, steps=3):
    """The differentiable batch (1024 problems, N = 256, n = 16, m = 8): the forward pass, and forward
    plus backward through the autograd.Function, loss sum ||x - x_ref||^2 + ||u||^2."""
    import numpy as np
    import torch
    from paper_2407_05433_gb300 import eclqr, synth
    from paper_2407_05433_gb300 import autograd as ag
    pbs = [synth.config("diff_batch", index=j) for j in range(1024)]
    b = eclqr.Batch(pbs, device=dev)
    try:
        b.run()
        fwd = statistics.median(_time_runs(b, steps, flush, stream))
        res = b.resid.cpu().numpy()
        stat = b.status.cpu().numpy()
        rng = np.random.default_rng(0)
        xref = torch.from_numpy(rng.standard_normal(int(b.layout.x))).to(dev)
        params = ag.batch_params(b)
        times = []
        for k in range(steps + 1):
            for p in params:
                p.grad = None
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            x, u = ag.solve(b, *params)
            loss = ((x - xref) ** 2).sum() + (u ** 2).sum()
            loss.backward()
            e1.record(stream)
            torch.cuda.synchronize()
            if k:
                times.append(e0.elapsed_time(e1))
        fb = statistics.median(times)
    finally:
        b.close()
    # checkpointed: four segments of 256 problems on one segment-sized handle, factors recomputed
    seg = eclqr.Batch(pbs[:256], device=dev)
    try:
        full = eclqr.Batch(pbs, device=dev)
        params = ag.batch_params(full)
        full.close()
        times = []
        for k in range(steps + 1):
            for p in params:
                p.grad = None
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            x, u = ag.solve_checkpointed(seg, 4, *params)
            (((x - xref) ** 2).sum() + (u ** 2).sum()).backward()
            e1.record(stream)
            torch.cuda.synchronize()
            if k:
                times.append(e0.elapsed_time(e1))
        fbc = statistics.median(times)
    finally:
        seg.close()
    stages = sum(p.N for p in pbs)
    return {"workload": "diff_batch: 1024 problems, N=256, n=16, m=8, 4 mixed rows, 4 terminal rows",
            "forward": {"value": stages / (fwd * 1e-3), "unit": "stages/s", "ms_per_step": fwd,
                        "resid_max": float(res.max()), "passed_at_1e-9": int(((stat == 0) & (res <= KKT_GATE)).sum())},
            "forward_backward": {"value": stages / (fb * 1e-3), "unit": "stages/s", "ms_per_step": fb},
            "forward_backward_checkpointed": {"value": stages / (fbc * 1e-3), "unit": "stages/s", "ms_per_step": fbc,
                                              "segments": 4, "note": "one 256-problem handle; factors recomputed "
                                                                     "in the backward pass"}}


def measure_scan_skip(dev, flush, stream, steps=3):
    """The Sec. 6 shortcut on mixed_only_n12 (N=1024, n=12, m=6, mixed rows U{0..4}, no state-only or
    terminal rows), with the shortcut and with the scan forced; both must give the same results."""
    import numpy as np
    from paper_2407_05433_gb300 import eclqr, synth
    pb = synth.config("mixed_only_n12")
    out, ref = {"workload": "mixed_only_n12: N=1024, n=12, m=6, mixed rows U{0..4}, no state-only or terminal rows"}, None
    for name, flag in (("skip", 1), ("scan", 0)):
        b = eclqr.Batch([pb], device=dev, scan_skip=flag)
        try:
            b.run()
            ms = statistics.median(_time_runs(b, steps, flush, stream))
            (r,) = b.results()
            skipped = bool(b.scan_skipped()[0])
        finally:
            b.close()
        out[name] = {"value": pb.N / (ms * 1e-3), "unit": "stages/s", "ms_per_step": ms, "scan_skipped": skipped,
                     "kkt_resid": r["resid"], "gate_passed": r["status"] == 0 and r["resid"] <= KKT_GATE}
        if ref is None:
            ref = r
        else:
            out["bit_identical"] = all(np.array_equal(np.asarray(ref[k]), np.asarray(r[k]))
                                       for k in ("x", "u", "lam", "mu", "eta", "alpha"))
    out["speedup"] = out["scan"]["ms_per_step"] / out["skip"]["ms_per_step"]
    return out


# ---------------------------------------------------------------- CPU oracle
def _oracle_worker(args):
    idx, seconds = args
    import oracle
    from paper_2407_05433_gb300 import synth
    pbs = [synth.config(WORKLOAD, index=j) for j in idx]
    for pb in pbs:
        oracle.solve(pb)
    stages, spent, t0 = 0, 0.0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        for pb in pbs:
            t = time.perf_counter()
            s = oracle.solve(pb)
            oracle.kkt_residual(pb, s.x, s.u, s.lam, s.mu, s.eta, s.alpha)
            spent += time.perf_counter() - t
            stages += pb.N
    return stages, spent


def host_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def oracle_rate(seconds, cores, sample=256):
    """The oracle as it stands on the host's cores over a bounded sample of the batch: draws
    0..sample-1 split over `cores` processes, each solving its share repeatedly for ~seconds; the rate
    is the sum of the per-process rates."""
    import multiprocessing as mp
    import oracle
    oracle.build_oracle()
    shares = [list(range(w, sample, cores)) for w in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        out = pool.map(_oracle_worker, [(s, seconds) for s in shares])
    rate = sum(st / sp for st, sp in out if sp > 0)
    return {"value": rate, "unit": "stages/s", "cores": cores, "kind": "oracle",
            "sample": f"draws 0..{sample - 1} of the batch split over {cores} processes, each solving its share "
                      f"(solve with refinement + residual) repeatedly for ~{seconds:.0f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    cores = host_cores()
    seconds = max(2.0, min(20.0, 2.0 * args.steps))
    cpu = oracle_rate(seconds, cores)
    value = cpu["value"]
    total = workload_flops().get(WORKLOAD, {}).get("stages") or 1076944
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "stages/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC, "problems": PROBLEMS},
            "cpu_baseline": {"value": value, "unit": "stages/s", "cores": cores, "kind": "oracle",
                             "sample": cpu["sample"]},
            "e2e": {"value": value, "unit": "stages/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- the GPU arm
def run_gpu(args):
    import numpy as np
    rank, world, local = dist_env()
    t_gen = time.perf_counter()
    draws, pbs = batched_problems(args.problems, args.state_dim, args.max_horizon)  # host-side, before any CUDA call
    t_gen = time.perf_counter() - t_gen
    fg = floor_gates()
    gates = {pos: fg[j] for pos, j in enumerate(draws) if j in fg}
    import torch
    from paper_2407_05433_gb300 import eclqr
    from paper_2407_05433_gb300 import build as build_mod

    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if rank == 0:
        build_mod.build()
    if world > 1:
        torch.distributed.barrier()
    build_mod.build()
    eclqr.load()
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2
    stages = int(sum(p.N for p in pbs))

    # untimed setup: the fewest refinement passes on the KKT residual that leave as many problems
    # under their gate as the library default (8), for one or two reduced passes in the first
    # solve; a captured step records every pass, so passes that no problem needs still cost their
    # launches and the sweeps of slow-converging problems
    refine, kkt_refine, kr_trials = autotune_refine(pbs, dev, gates, flush, stream, team_warps=args.team_warps)
    batch = eclqr.Batch(pbs, device=dev, refine=refine, corr_refine=CORR_REFINE, kkt_refine=kkt_refine,
                        team_warps=args.team_warps)
    per_replay = batch.capture()            # eager pass on a side stream, then one captured pass
    for _ in range(max(3, args.warmup)):
        batch.replay()
    torch.cuda.synchronize(dev)

    # timed region: graph replays, L2 flushed between them (outside the events)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    step_ms = _time_replays(batch, args.steps, flush, stream)
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    ms = total_ms / args.steps
    res = batch.resid.cpu().numpy()
    stat = batch.status.cpu().numpy()
    passed, gate = gate_report(pbs, res, stat, gates)
    solved = int(sum(p.N for p, ok in zip(pbs, passed) if ok))
    solved = sum_over_ranks(solved, world, dev)
    all_ok = all_ranks(bool(passed.all()), world, dev)
    value = solved / (ms * 1e-3)

    # end to end through the public API with host buffers: pinned H2D of every input, the four
    # calls (eager), D2H of every output, all inside the timed region
    host_in = {k: torch.from_numpy(batch.host[k]).pin_memory() for k in eclqr.DATA_KEYS + ("s0",)}
    outs = ("x", "u", "lam", "mu", "eta", "alpha", "resid", "status")
    host_out = {k: torch.empty_like(getattr(batch, k), device="cpu").pin_memory() for k in outs}
    h2d = sum(t.numel() * t.element_size() for t in host_in.values())
    d2h = sum(t.numel() * t.element_size() for t in host_out.values())

    def e2e_step():
        for k, t in host_in.items():
            batch.d[k].copy_(t, non_blocking=True)
        batch.run()
        for k in outs:
            host_out[k].copy_(getattr(batch, k), non_blocking=True)

    e2e_step()
    torch.cuda.synchronize(dev)
    e2e_steps = max(2, min(5, args.steps // 4))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_ms = 0.0
    for _ in range(e2e_steps):
        flush.zero_()
        ev0.record(stream)
        e2e_step()
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        e2e_ms += ev0.elapsed_time(ev1)
    e2e_ms = max_over_ranks(e2e_ms / e2e_steps, world, dev)
    e_passed, _ = gate_report(pbs, host_out["resid"].numpy(), host_out["status"].numpy(), gates)
    e2e_solved = sum_over_ranks(int(sum(p.N for p, ok in zip(pbs, e_passed) if ok)), world, dev)

    if rank != 0:
        batch.close()
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    flops_all = workload_flops()
    # the oracle's count for the same number of reduced refinement passes in the first solve
    fl = flops_all.get(WORKLOAD + ("" if refine == 2 else "_refine%d" % refine)) if (
        args.problems == PROBLEMS and args.state_dim is None and args.max_horizon is None) else None
    peak = eclqr.eclqr_probe_fp64_peak()
    extras = {}
    kern = None
    if not args.no_extra:
        extras["plain"] = measure_plain(pbs, dev, flush, stream)
        extras["plain"]["speedup_batched_vs_plain"] = value / extras["plain"]["value"]
        kern = measure_kernels(pbs, dev, flush, stream, fl, refine)
        extras["kernels"] = kern
        extras["without_kkt_refine"] = measure_without_kkt_refine(pbs, dev, flush, stream, gates, refine)
    batch.close()
    roofline = None
    if fl:
        step_flops = fl["step_flops"]
        roofline = {"bound": "alu", "unit": "TFLOP/s", "peak": peak,
                    "peak_source": "FP64 FMA throughput measured on this GPU by eclqr_probe_fp64_peak (no FP64 "
                                   "entry in MEASURED_PEAKS.json)",
                    "step_achieved": step_flops / (ms * 1e-3) / 1e12,
                    "step_frac": step_flops / (ms * 1e-3) / 1e12 / peak,
                    "step_algorithmic_flops": step_flops, "traffic": None}
        if kern and "phase_kernels" in kern:
            pk = {k: v for k, v in kern["phase_kernels"].items() if v["ms"]}
            dom = max(pk, key=lambda k: pk[k]["ms"])
            d = pk[dom]
            achieved = d["achieved_tflops"]
            roofline.update({"kernel": dom, "achieved": achieved, "frac": achieved / peak,
                             "kernel_ms_per_step": d["ms"], "algorithmic_flops_per_step": d["algorithmic_flops"],
                             "launches_per_step": kern["launches_per_step"].get(dom)})
            tpath = os.path.join(ROOT, "profiles", "dram_traffic.json")
            if os.path.exists(tpath):
                try:
                    t = json.load(open(tpath))
                    if t.get("kernel") == dom and t.get("workload") == WORKLOAD:
                        roofline["traffic"] = t.get("bytes_per_launch")
                except (OSError, ValueError):
                    pass
        else:
            roofline.update({"achieved": roofline["step_achieved"], "frac": roofline["step_frac"]})
    if world == 1 and not args.no_extra:
        from paper_2407_05433_gb300 import synth
        extras["long_n16"] = single_line("long_n16: N=65536, n=16, m=8, 4 mixed rows, terminal rank 8, A orthogonal",
                                         synth.config("long_n16"), dev, flush, stream, 2)
        extras["degenerate_n12"] = single_line("degenerate_n12: N=1024, n=12, m=6, mixed rows U{0..8}, 20% degenerate "
                                               "stages, full-rank terminal", synth.config("degenerate_n12"), dev,
                                               flush, stream, 5)
        extras["single_n4"] = single_line("single_n4: N=64, n=4, m=2, 1 mixed row, rank-2 terminal",
                                          synth.config("single_n4"), dev, flush, stream, 5)
        for key in ("degenerate_n12", "single_n4"):   # the plain solve of the same instance: one chunk
            pb = synth.config(key)
            extras[key]["plain"] = single_line(key + " as one chunk", pb, dev, flush, stream, 3, chunk=pb.N)
        extras["table1"] = [single_line(f"table1: N={N}, n=8, m=4, 2 state-only rows per nonterminal stage",
                                        synth.config("table1", N=N), dev, flush, stream, 3)
                            for N in (1024, 4096, 16384)]
        extras["diff_batch"] = measure_diff_batch(dev, flush, stream)
        extras["scan_skip"] = measure_scan_skip(dev, flush, stream)
        extras["mixed"] = {
            "long_n16": measure_mixed("long_n16: N=65536, n=16, m=8", [synth.config("long_n16")], dev, flush, stream),
            "diff_batch": measure_mixed("diff_batch: 1024 problems, N=256, n=16, m=8",
                                        [synth.config("diff_batch", index=j) for j in range(1024)], dev, flush,
                                        stream),
            "single_n4": measure_mixed("single_n4: N=64, n=4, m=2", [synth.config("single_n4")], dev, flush,
                                       stream, steps=5),
            "batched_uneven": measure_mixed("batched_uneven: the headline batch, graph replay", pbs, dev, flush,
                                            stream, gates=gates, graph=True),
        }
        for key, wk in (("long_n16", "long_n16"), ("degenerate_n12", "degenerate_n12"), ("single_n4", "single_n4")):
            f = flops_all.get(wk)
            if f:
                extras[key]["step_frac_fp64"] = f["step_flops"] / (extras[key]["ms_per_step"] * 1e-3) / 1e12 / peak
    cpu = None
    if args.cpu_seconds > 0 and world == 1:
        cpu = oracle_rate(args.cpu_seconds, host_cores())
    line = {
        "metric": METRIC, "value": value, "unit": "stages/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "problems_per_gpu": len(pbs), "stages_per_gpu": stages,
                   "l2": f"inputs of {h2d / 1e9:.1f} GB per GPU (larger than L2); a 256 MB buffer is also written "
                         "between steps",
                   "team_warps": args.team_warps or "per kernel", "state_dim": args.state_dim,
                   "max_horizon": args.max_horizon,
                   "step": "graph replay of eclqr_build + eclqr_solve + eclqr_multipliers + eclqr_refine",
                   "refine": refine, "corr_refine": CORR_REFINE, "kkt_refine": kkt_refine,
                   "refine_autotune": kr_trials,
                   "refine_tol": 5e-10, "generation_s": round(t_gen, 1)},
        "gate": gate, "gate_passed": all_ok,
        "e2e": {"value": e2e_solved / (e2e_ms * 1e-3), "unit": "stages/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                "call": "Batch.run (eager) with pinned host copies of every input and output"},
        "gpu_launches": per_replay * args.steps,
        "launches_per_step": per_replay,
        "roofline": roofline,
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    line.update(extras)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--problems", type=int, default=PROBLEMS, help="draws 0..problems-1 of the batch")
    ap.add_argument("--state-dim", type=int, default=None,
                    help="keep only the draws with this state dimension (one (n, m) group, for profiling)")
    ap.add_argument("--max-horizon", type=int, default=None,
                    help="cap the horizons (a smaller case of the same shape, for profiling)")
    ap.add_argument("--team-warps", type=int, default=0,
                    help="warps per task for every kernel (0: the library's per-kernel choice)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-extra", action="store_true", help="skip the plain solve, kernel times and other workloads")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
