#!/usr/bin/env python
"""Throughput benchmark: equality-constrained LQR stages solved per second.

One step is one pass of the whole path of Algorithm 1 over one problem
instance through the C ABI: eclqr_build (suffix-domain scan, stage
elimination, Riccati factors), eclqr_solve (rollout with refinement and
recovery of x, u), eclqr_multipliers (Sec. 7) and eclqr_kkt_residual (the
Sec. 9 residual, the gate of the metric).  The workload is the degenerate
n = 12 instance (N = 1024, m = 6, mixed rows U{0..8} per stage, 20% of stages
with duplicated or D = 0 rows, full-rank terminal rows), seeded and synthetic.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference] [--no-extra]

At N = 1 the line also carries "graph" (the same step captured once into a
CUDA graph and replayed), "plain" (the same instance as one chunk: a single
CTA sweeps every stage, no scan), "scan_skip" (the Sec. 6 shortcut on an
instance without state-only or terminal rows, with and without the skip) and
"batched" (4096 uneven problems, a
stand-in for the batched configuration, with the oracle on all host cores
beside it).

Under torchrun every rank solves its own copy (weak scaling, no collective on
the data path); rank 0 prints one JSON line.  ``--impl reference`` times the
CPU oracle on the host instead (rank 0 only).
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
WORKLOAD = "degenerate_n12"
WORKLOAD_DESC = ("degenerate_n12: one instance, N=1024, n=12, m=6, mixed rows U{0..8} per stage, 20% of stages "
                 "with duplicated or D=0 rows, full-rank terminal rows, A=I+0.1 randn, seed 0")
KKT_GATE = 1e-9
KERNELS = ["k_terminal", "k_primal_up", "k_rel_level", "k_primal_down", "k_param", "k_elim", "k_lqr_up",
           "k_lqr_level", "k_riccati_down", "k_aff_up", "k_aff_level", "k_aff_down", "k_solve_init",
           "k_post_roll", "k_resid", "k_pcorr", "k_recover", "k_dual_stage", "k_dual_terminal", "k_dual_up",
           "k_dual_down", "k_dual_root", "k_dual_leaf", "k_kkt_residual"]
# phase of Algorithm 1 each kernel implements (index into the oracle's per-phase flop counts)
KERNEL_PHASE = {"k_terminal": 0, "k_primal_up": 0, "k_rel_level": 0, "k_primal_down": 0, "k_param": 1,
                "k_elim": 2, "k_lqr_up": 3, "k_lqr_level": 3, "k_riccati_down": 3, "k_aff_up": 4,
                "k_aff_level": 4, "k_aff_down": 4, "k_solve_init": 4, "k_post_roll": 4, "k_resid": 4,
                "k_pcorr": 4, "k_recover": 4, "k_dual_stage": 5, "k_dual_terminal": 5, "k_dual_up": 5,
                "k_dual_down": 5, "k_dual_root": 5, "k_dual_leaf": 5, "k_kkt_residual": 6}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


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


def job_rate(world, stages_per_rank, ms):
    """Whole-job throughput: every rank solves its own copy (weak scaling) within the slowest rank's time."""
    return world * stages_per_rank / (ms * 1e-3)


def oracle_rate(pb, seconds):
    """The CPU oracle as it stands, one thread, repeated over the workload for ~seconds."""
    import oracle
    oracle.build_oracle()
    oracle.solve(pb)  # warm
    n, t0 = 0, time.perf_counter()
    times = []
    while True:
        t = time.perf_counter()
        s = oracle.solve(pb)
        oracle.kkt_residual(pb, s.x, s.u, s.lam, s.mu, s.eta, s.alpha)
        times.append(time.perf_counter() - t)
        n += 1
        if time.perf_counter() - t0 > seconds:
            break
    return pb.N / statistics.median(times), n, statistics.median(times)


def _timed_runs(batch, steps, flush, stream):
    """Device time per full pass (build, solve, multipliers, residual) with L2 flushed between passes."""
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
    return statistics.median(times)


def measure_graph(batch, pb, flush, stream, steps):
    """The same step captured once into a CUDA graph and replayed (same kernels, same order)."""
    import torch
    nl = batch.capture()
    for _ in range(3):
        batch.replay()
    times = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = statistics.mean(times)
    (r,) = batch.results()
    return {"value": pb.N / (ms * 1e-3), "unit": "stages/s", "ms_per_step": ms, "launches_per_replay": nl,
            "kkt_resid": r["resid"], "gate_passed": r["status"] == 0 and r["resid"] <= KKT_GATE}


def measure_plain(pb, dev, flush, stream, refine, steps=3):
    """The plain GPU solve: one chunk spanning the horizon, so a single CTA per problem sweeps every stage
    in order (no scan), beside the chunked scan form of the main line."""
    from paper_2407_05433_gb300 import eclqr
    b = eclqr.Batch([pb], device=dev, refine=refine, chunk=pb.N)
    b.run()
    ms = _timed_runs(b, steps, flush, stream)
    (r,) = b.results()
    b.close()
    return {"value": pb.N / (ms * 1e-3), "unit": "stages/s", "ms_per_step": ms, "chunk": pb.N,
            "kkt_resid": r["resid"], "status": r["status"], "gate_passed": r["status"] == 0 and r["resid"] <= KKT_GATE}


def measure_scan_skip(dev, flush, stream, refine, steps=5):
    """The Sec. 6 shortcut on an instance it applies to: mixed_only_n12 (N=1024, n=12, m=6, mixed rows
    U{0..4} per stage with wide full-row-rank D_i, no state-only or terminal rows), timed with the shortcut
    (domain scan skipped) and without it (scan forced).  Both passes must give the same results."""
    import numpy as np
    from paper_2407_05433_gb300 import eclqr, synth
    pb = synth.config("mixed_only_n12")
    out, ref = {"workload": "mixed_only_n12: N=1024, n=12, m=6, mixed rows U{0..4}, no state-only or terminal rows"}, None
    for name, flag in (("skip", 1), ("scan", 0)):
        b = eclqr.Batch([pb], device=dev, refine=refine, scan_skip=flag)
        b.run()
        ms = _timed_runs(b, steps, flush, stream)
        (r,) = b.results()
        skipped = bool(b.scan_skipped()[0])
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


BATCH_DISTINCT, BATCH_PROBLEMS = 256, 4096


def batched_problems():
    from paper_2407_05433_gb300 import synth
    base = [synth.config("batched_uneven", index=j) for j in range(BATCH_DISTINCT)]
    return base, [base[j % BATCH_DISTINCT] for j in range(BATCH_PROBLEMS)]


def measure_batched(pbs, dev, flush, stream, refine, steps=3):
    """Config 4 stand-in: 4096 uneven problems (256 seeded draws of the generator, each repeated 16 times)
    solved as one batch through the same calls."""
    import numpy as np
    from paper_2407_05433_gb300 import eclqr
    b = eclqr.Batch(pbs, device=dev, refine=refine)
    b.run()
    ms = _timed_runs(b, steps, flush, stream)
    res = b.resid.cpu().numpy()
    stat = b.status.cpu().numpy()
    launches = b.launches()
    skipped = int(b.scan_skipped().sum())
    # per-kernel device time over one untimed pass each; the (n, m) groups run concurrently on their
    # own streams, so a kernel's time is summed over its groups' overlapping launches
    kernel_ms = {}
    try:
        for name in KERNELS + ["k_scan_check"]:
            eclqr.eclqr_time_kernel(b.h, name)
            b.run()
            nl, tms = eclqr.eclqr_kernel_time(b.h)
            if nl:
                kernel_ms[name] = round(tms, 3)
    except Exception as exc:  # informative only: never lose the line for it
        kernel_ms = {"error": str(exc)}
    finally:
        eclqr.eclqr_time_kernel(b.h, None)
    b.close()
    stages = int(sum(p.N for p in pbs))
    passed = (stat == 0) & (res <= KKT_GATE)
    return {"value": stages / (ms * 1e-3), "unit": "stages/s", "ms_per_step": ms, "problems": len(pbs),
            "stages": stages, "distinct_draws": BATCH_DISTINCT, "refine": refine,
            "status_failures": int((stat != 0).sum()), "resid_max": float(res.max()),
            "gate_passed_frac": float(passed.mean()), "gate_passed": bool(passed.all()),
            "scan_skipped_problems": skipped, "kernel_ms_per_pass_summed_over_groups": kernel_ms}


def _oracle_worker(args):
    idx, seconds = args
    import oracle
    from paper_2407_05433_gb300 import synth
    pbs = [synth.config("batched_uneven", index=j) for j in idx]
    for pb in pbs:
        oracle.solve(pb)
    stages, spent, t0 = 0, 0.0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        for pb in pbs:
            t = time.perf_counter()
            oracle.solve(pb)
            spent += time.perf_counter() - t
            stages += pb.N
    return stages, spent


def oracle_batched_rate(seconds, cores):
    """The oracle on the host's cores over a bounded sample of the batch: every process solves its own
    share of the 256 draws repeatedly for ~seconds; the rate is the sum of the per-process rates."""
    import multiprocessing as mp
    import oracle
    oracle.build_oracle()
    shares = [list(range(w, BATCH_DISTINCT, cores)) for w in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        out = pool.map(_oracle_worker, [(s, seconds) for s in shares])
    rate = sum(st / sp for st, sp in out if sp > 0)
    return {"value": rate, "unit": "stages/s", "cores": cores, "kind": "oracle",
            "sample": f"the {BATCH_DISTINCT} distinct draws split over {cores} processes, each solving its share "
                      f"repeatedly for ~{seconds:.0f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2407_05433_gb300 import synth
    import oracle
    oracle.build_oracle()
    pb = synth.config(WORKLOAD)
    for _ in range(args.warmup):
        oracle.solve(pb)
    times, resid = [], None
    for _ in range(args.steps):
        t = time.perf_counter()
        s = oracle.solve(pb)
        resid = oracle.kkt_residual(pb, s.x, s.u, s.lam, s.mu, s.eta, s.alpha)
        times.append(time.perf_counter() - t)
    ms = 1e3 * statistics.mean(times)
    value = pb.N / (ms * 1e-3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "stages/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC, "stages": pb.N, "kkt_resid": resid, "status": s.status},
            "cpu_baseline": {"value": value, "unit": "stages/s", "cores": 1, "kind": "oracle",
                             "sample": f"the full workload ({pb.N} stages) per step, one thread"},
            "e2e": {"value": value, "unit": "stages/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import numpy as np
    import torch
    from paper_2407_05433_gb300 import eclqr, synth
    from paper_2407_05433_gb300 import build as build_mod

    rank, world, local = dist_env()
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

    pb = synth.config(WORKLOAD)
    chunk, trials = args.chunk, None
    if chunk == 0:
        # untimed setup: the fastest chunk length whose pass meets the residual gate
        chunk, trials = eclqr.autotune_chunk([pb], device=dev, refine=args.refine, gate=KKT_GATE)
    batch = eclqr.Batch([pb], device=dev, refine=args.refine, chunk=chunk)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2

    def step():
        batch.build()
        batch.solve()
        batch.multipliers()
        batch.residual()

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize(dev)

    # which kernel dominates the step: bracket each kernel in turn over one untimed step
    per_kernel = {}
    for name in KERNELS:
        eclqr.eclqr_time_kernel(batch.h, name)
        step()
        nl, tms = eclqr.eclqr_kernel_time(batch.h)
        per_kernel[name] = (nl, tms)
    eclqr.eclqr_time_kernel(batch.h, None)
    dominant = max(per_kernel, key=lambda k: per_kernel[k][1])

    # timed region: per-step events, L2 flushed between steps (outside the events)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    eclqr.eclqr_time_kernel(batch.h, dominant)
    launches0 = batch.launches()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    for k in range(args.steps):
        flush.zero_()
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
    torch.cuda.synchronize(dev)
    launches = batch.launches() - launches0
    nl_dom, t_dom = eclqr.eclqr_kernel_time(batch.h)
    eclqr.eclqr_time_kernel(batch.h, None)
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = sum(step_ms)
    total_ms = max_over_ranks(total_ms, world, dev)
    (res,) = batch.results()
    ok = all_ranks(res["status"] == 0 and res["resid"] <= KKT_GATE, world, dev)

    # end to end through the C ABI with host buffers: pinned H2D of the inputs,
    # the four calls, D2H of every output, all inside the timed region
    host_in = {k: torch.from_numpy(batch.host[k]).pin_memory() for k in eclqr.DATA_KEYS + ("s0",)}
    outs = ("x", "u", "lam", "mu", "eta", "alpha", "resid", "status")
    host_out = {k: torch.empty_like(getattr(batch, k), device="cpu").pin_memory() for k in outs}
    h2d = sum(t.numel() * t.element_size() for t in host_in.values())
    d2h = sum(t.numel() * t.element_size() for t in host_out.values())
    e2e_steps = max(5, args.steps // 4)

    def e2e_step():
        for k, t in host_in.items():
            batch.d[k].copy_(t, non_blocking=True)
        step()
        for k in outs:
            host_out[k].copy_(getattr(batch, k), non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize(dev)
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
    e2e_ok = all_ranks(int(host_out["status"][0]) == 0 and float(host_out["resid"][0]) <= KKT_GATE, world, dev)

    if rank != 0:
        batch.close()
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    extras = {}
    if world == 1 and not args.no_extra:
        extras["graph"] = measure_graph(batch, pb, flush, stream, max(5, args.steps // 2))
        extras["plain"] = measure_plain(pb, dev, flush, stream, args.refine)
        extras["scan_skip"] = measure_scan_skip(dev, flush, stream, args.refine)
        _, bpbs = batched_problems()
        extras["batched"] = measure_batched(bpbs, dev, flush, stream, args.refine)
    import oracle
    oracle.build_oracle()
    sref = oracle.solve(pb)
    phase = sref.phase_flops
    step_flops = float(np.sum(phase[:6]))
    ms = total_ms / args.steps
    value = job_rate(world, pb.N, ms)
    peak = eclqr.eclqr_probe_fp64_peak()
    dom_ms = t_dom / max(1, nl_dom)
    launches_per_step_dom = nl_dom / args.steps
    dom_flops = phase[KERNEL_PHASE[dominant]] / max(1.0, launches_per_step_dom)
    achieved = dom_flops / (dom_ms * 1e-3) / 1e12
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if os.path.exists(tpath):
        try:
            tinfo = json.load(open(tpath))
            if tinfo.get("kernel") == dominant and tinfo.get("workload") == WORKLOAD:
                traffic = tinfo.get("bytes_per_launch")
        except (OSError, ValueError):
            traffic = None
    cpu = None
    if args.cpu_seconds > 0:
        rate, nrun, med = oracle_rate(pb, args.cpu_seconds)
        cpu = {"value": rate, "unit": "stages/s", "cores": 1, "kind": "oracle",
               "sample": f"full workload ({pb.N} stages) solved {nrun} times in ~{args.cpu_seconds:.0f} s, "
                         f"median {med * 1e3:.1f} ms per solve, one thread"}
    line = {
        "metric": METRIC, "value": value if ok else 0.0, "unit": "stages/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "stages_per_gpu": pb.N, "refine": args.refine,
                   "chunk": chunk, "chunk_autotune": [{"chunk": c, "ms": round(t, 3), "kkt_resid": r, "passed": ok}
                                                      for c, t, r, ok in (trials or [])],
                   "l2": "256 MB buffer written between timed steps",
                   "kkt_resid": res["resid"], "status": res["status"], "gate_passed": ok,
                   "step": "eclqr_build + eclqr_solve + eclqr_multipliers + eclqr_kkt_residual"},
        "e2e": {"value": job_rate(world, pb.N, e2e_ms) if e2e_ok else 0.0, "unit": "stages/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "kernel": dominant, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "avg_launch_ms": dom_ms, "launches_per_step": launches_per_step_dom,
                     "algorithmic_flops_per_launch": dom_flops,
                     "peak_source": "FP64 FMA probe (eclqr_probe_fp64_peak) on this GPU",
                     "step_achieved": step_flops / (ms * 1e-3) / 1e12,
                     "step_frac": step_flops / (ms * 1e-3) / 1e12 / peak},
        "kernel_ms_per_step": {k: round(v[1], 4) for k, v in per_kernel.items()},
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    line.update(extras)
    if "batched" in extras and args.cpu_seconds > 0:
        cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
        line["batched"]["cpu_baseline"] = oracle_batched_rate(args.cpu_seconds, cores)
    print(json.dumps(line), flush=True)
    batch.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--refine", type=int, default=2)
    ap.add_argument("--chunk", type=int, default=0, help="stages per scan chunk; 0 = autotuned (untimed setup)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-extra", action="store_true", help="skip the plain-solve and batched lines")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
