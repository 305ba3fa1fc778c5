"""Oracle: plain, slow, obviously correct FP64 CPU reference.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product path (the CUDA library under ``paper_1510_03110_gb300``) shares no code
with it and never calls it.

Modules
  core   ctypes binding of ``uftoc_oracle.c`` (serial Riccati, Algorithms 1-3;
         MHE stage assembly, Section II; KKT residual; objective) and the
         generic UFTOC container.
  dense  dense KKT assembly + LAPACK LU solve (the Newton step by definition).
  rts    Kalman filter + Rauch-Tung-Striebel smoother (textbook), used to pin
         the MHE -> UFTOC transform.
  boxqp  MHE with box-bounded process noise (Section II's constrained MHE),
         solved exactly by a primal active-set method on the dense KKT system.
  tree   the paper's parallel scheme executed serially: Algorithm 4 (chunk
         reduction), the master problem (Section IV-C), Algorithms 5 and 6.
"""
from .core import (Uftoc, mhe_to_uftoc, riccati, kkt_residual, objective,  # noqa: F401
                   mhe_stage, split_solution, relres)
