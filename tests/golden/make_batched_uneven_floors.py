"""Writes batched_uneven_floors.txt: the FP64 residual floor of every draw of the uneven-batch
workload (problems 0..4095 of synth.config("batched_uneven")) whose floor can reach the 1e-9 gate.

The floor belongs to the problem, not to a method.  The exact KKT solution w* (oracle.exact:
sparse LU with extended-precision refinement of the Sec. 2 problem's KKT system) is rounded to
FP64, and every row of the residual (Sec. 9 definition) of such a point moves by a small multiple
of the unit roundoff times the row's scale |K||w| + |b|.  The file lists, per draw,

    rho   the Sec. 9 residual of the rounded exact solution, evaluated in FP64 by the oracle
    phi   eps * max over rows of |K||w*| + |b| (eps = 2^-52)
    ext   the extended-precision residual of w* before rounding: about 1e-16 or less where the
          refinement converged; far above it the KKT matrix is too close to singular for w* (and
          phi) to be trusted

for every draw with 4 * phi > 1e-9.  A draw listed here is gated at max(1e-9, 4 * phi); every
other draw at 1e-9.  Only oracle/ and the input generator are used:

    python tests/golden/make_batched_uneven_floors.py [--problems 4096] [--procs 8]
"""
from __future__ import annotations

import argparse
import os
import sys
from multiprocessing import get_context

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "batched_uneven_floors.txt")
GATE = 1e-9
FACTOR = 4.0


def _floor(j):
    import numpy as np
    import oracle
    from oracle.exact import exact_kkt, residual_scale
    from paper_2407_05433_gb300 import synth
    eps = float(np.finfo(float).eps)
    pb = synth.config("batched_uneven", index=j)
    e = exact_kkt(pb)
    rho = oracle.kkt_residual(pb, e["x"], e["u"], e["lam"], e["mu"], e["eta"], e["alpha"])
    phi = eps * float(residual_scale(pb, e).max())
    return j, pb.N, pb.n, rho, phi, e["ext_resid"]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--problems", type=int, default=4096)
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    import oracle
    oracle.build_oracle()
    with get_context("spawn").Pool(args.procs) as pool:
        rows = pool.map(_floor, range(args.problems), chunksize=4)
    with open(OUT, "w") as f:
        f.write("# FP64 residual floors of the uneven-batch draws (synth.config('batched_uneven', index=j)),\n")
        f.write(f"# problems 0..{args.problems - 1}; written by make_batched_uneven_floors.py from oracle/ only.\n")
        f.write(f"# Listed: draws with {FACTOR:g} * phi > {GATE:g}; their gate is max({GATE:g}, {FACTOR:g} * phi).\n")
        f.write("# index N n rho phi ext\n")
        for j, N, n, rho, phi, ext in rows:
            if FACTOR * phi > GATE:
                f.write(f"{j} {N} {n} {rho:.6e} {phi:.6e} {ext:.3e}\n")


if __name__ == "__main__":
    main()
