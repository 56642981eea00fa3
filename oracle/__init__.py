"""Plain FP64 CPU oracle for decoupled multicontinuum time stepping
(Vasilyeva, "Efficient decoupling schemes for multiscale multicontinuum
problems in fractured porous media", arXiv 2209.01158).

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or
execute this package: only the tests, the smoke check and the benchmark's
CPU-baseline leg use it. It shares no code with the CUDA path; both consume
the same seeded inputs from `mc_inputs`.

Every step is the plain definition written out: assemble the finite-volume
matrices of Section 3.1 as scipy sparse matrices and solve each time step's
linear system with a sparse direct factorisation (SuperLU) plus FP64
iterative refinement. Nothing is blocked, fused or reordered.

Modules:
  fv       -- TPFA assembly of M, D_alpha, Q_alpha_beta, F (Section 3.1).
  schemes  -- coupled backward Euler (Eq. ct-mc) and the decoupled D-, L-,
              U-schemes (Eq. si-mc, Section 3.3).
  nlmc     -- NLMC multiscale basis (Eq. eq:basis), R, A_bar = R A R^T and the
              coarse coupled / decoupled schemes (Section 4).
  metrics  -- relative L2 errors e_h, e_H (Section 5), mass and energy.

Parity status of each function is stated in its docstring; all are pinned by
the CPU tests (closed forms, invariants, dense brute force, special cases).
"""

from .fv import FVSystem, harmonic_face
from .schemes import Oracle
from .nlmc import NLMC
from . import metrics

__all__ = ["FVSystem", "harmonic_face", "Oracle", "NLMC", "metrics"]
