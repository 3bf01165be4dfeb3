"""Writes workload_flops.json: the algorithmic FP64 work of every benchmark workload, per phase.

The algorithmic work of a step is the oracle's own count (standard formulas: Householder step on
an r x c block 4rc, GEMM 2mnk, Cholesky n^3/3, triangular solve n^2 per right-hand side) for one
pass of the work-efficient sequential method: phases 0 suffix domains (Sec. 3-4), 1 domain
parameterisation, 2 stage elimination (Sec. 5), 3 Riccati factors (Sec. 6), 4 rollout,
refinement on the reduced residual and recovery, 5 multipliers (Sec. 7), 6 KKT residual (Sec. 9);
phase 7 is the refinement on the original KKT residual, counted separately and not as useful
work.  Scan overhead of the GPU path (chunk aggregates, compositions) is not counted.
"batched_uneven_refine1" is the uneven batch with one reduced refinement pass in phase 4
instead of two, the count the benchmark's autotuner may choose for the first solve.

    python tests/golden/make_workload_flops.py [--procs 8]

Only oracle/ and the input generator are used.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
from multiprocessing import get_context

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "workload_flops.json")


def _flops(job):
    import oracle
    from paper_2407_05433_gb300 import synth
    name, kw, refine = job
    pb = synth.config(name, **kw)
    s = oracle.solve(pb, refine=refine)
    return name + ("_refine%d" % refine if refine != 2 else ""), kw, pb.N, [float(v) for v in s.phase_flops] + [max(0.0, float(s.flops - sum(s.phase_flops)))]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    import oracle
    oracle.build_oracle()
    jobs = [("batched_uneven", {"index": j}, r) for r in (2, 1) for j in range(4096)]
    jobs += [("diff_batch", {"index": j}, 2) for j in range(1024)]
    jobs += [(k, {}, 2) for k in ("single_n4", "degenerate_n12", "long_n16", "mixed_only_n12")]
    jobs += [("table1", {"N": N}, 2) for N in (1024, 4096, 16384)]
    with get_context("spawn").Pool(args.procs) as pool:
        rows = pool.map(_flops, jobs, chunksize=8)
    out = {}
    for name, kw, N, ph in rows:
        key = name if name.startswith(("batched_uneven", "diff_batch")) else name + ("_N%d" % kw["N"] if "N" in kw else "")
        e = out.setdefault(key, {"problems": 0, "stages": 0, "phase_flops": [0.0] * 8})
        e["problems"] += 1
        e["stages"] += N
        e["phase_flops"] = [a + b for a, b in zip(e["phase_flops"], ph)]
    for e in out.values():
        e["step_flops"] = sum(e["phase_flops"][:7])
        e["flops_per_stage"] = e["step_flops"] / e["stages"]
    with open(OUT, "w") as f:
        json.dump({"note": "written by make_workload_flops.py from oracle/ only; phases 0-6 = one pass of the "
                           "sequential method (useful work), 7 = corrections of the refinement on the original "
                           "KKT residual", "workloads": out}, f, indent=1)


if __name__ == "__main__":
    main()
