"""CPU oracle for the space-time collocation / DG reaction-diffusion system.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 (numpy/scipy)
statement of what the GPU library computes, written from the paper
(Benedusi, Minion, Krause: "An experimental comparison of a space-time
multigrid method with PFASST for a reaction-diffusion problem", Sections 2-4).
Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the library never calls it, and it shares no code
with the CUDA path (inputs come from ``stgen``, which holds no solver
arithmetic).

Modules
  collocation  right Radau nodes, Q (Eq. 2.3-2.4), stability function, DG
               matrices (Eq. 2.8-2.10), time transfers, SDC Q_Delta
  space        FD / lumped-FEM Laplacians (Eq. 3.2), reaction terms (Eq. 3.1,
               3.7), spatial transfers (Section 5.2, SMG), grid coarsening
  system       the all-at-once residual G(U) (Eq. 2.3 with 2.11 and 3.4),
               linearisations, direct and sequential solves, DG solve
  multilevel   level operators, transfers and the exact coarse solve
  sdc          IMEX SDC sweep on the collocation problem (Section 4.1)
  adjoint      the transposed all-at-once system and gradients

Parity status: every function is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` except three helpers whose content is solver
design, not paper content - parity unpinned for
``multilevel.smoothing_step_exact`` (relaxation weight and block choice),
``multilevel.smoothing_step_jacobi`` (sweep count and weights) and
``multilevel.restrict_cbar_time`` (the slab average of the coarse levels'
reaction coefficient).  The slab transfers are pinned by the Galerkin
identity R_t (A_f - C_f) P_t = A_c - C_c.
"""
from . import collocation, space, system, multilevel, sdc, adjoint  # noqa: F401
