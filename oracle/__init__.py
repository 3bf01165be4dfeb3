"""CPU oracle for the equality-constrained LQR reduction (arXiv 2407.05433).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  It shares no code with
the CUDA path.

Two independent parts:
  * ``solve``      -- O2, the plain sequential FP64 reduction in C
                      (``eclqr_oracle.c``), following Algorithm 1 with the
                      sequential multiplier variant of Sec. 7.
  * ``dense_kkt``  -- O1, the plain definition: the unique minimiser of the QP
                      (Sec. 2, eq. problem) and its min-norm KKT multipliers,
                      from one dense least-squares solve of the KKT system.
"""
from .core import (solve, kkt_residual, build_oracle, load_mutant, OracleSolution, STATUS_NAMES,
                   project_rows, tqr_solve)
from .dense import dense_kkt, objective, brute_suffix_domain, constraint_matrix

__all__ = ["solve", "kkt_residual", "build_oracle", "load_mutant", "OracleSolution", "STATUS_NAMES",
           "project_rows", "tqr_solve", "dense_kkt", "objective", "brute_suffix_domain",
           "constraint_matrix"]
