"""Seeded synthetic test problems for the p-BiCGStab solver and its oracle.

This module only builds inputs (matrices, right-hand sides, initial guesses).
It holds none of the solver's arithmetic, so both the CUDA path and the CPU
oracle may use it.  Every generator is deterministic for a given seed
(numpy PCG64).

Stencils (all scaled by h^2, Dirichlet boundary nodes eliminated, row index
``(k*ny + j)*nx + i``):

* 2D Poisson 5-point (test problem TP1 of the paper, Table "tab:specs"):
  centre 4, neighbours -1.
* TP2 (Table "tab:specs"): 2D 5-point with the east and north couplings
  raised to -1+eps (the "upper triangular entries").
* 2D first-order upwind convection-diffusion, -Lap u + beta.grad u with
  beta = (1,1)/h * 0.5: centre 4 + h*bx + h*by = 5, west/south -1.5,
  east/north -1.
* 3D 7-point upwind convection-diffusion, beta = (1,0.5,0.25)/h * 0.8:
  centre 7.4, west -1.8, south -1.4, down -1.2, east/north/up -1.

Normalisation (Section 4 of the paper: the system matrix is rescaled to a unit
2-norm): the matrix is divided by sigma = sqrt(||A||_1 ||A||_inf), a cheap,
deterministic upper bound of ||A||_2 that is within 1e-3 of ||A||_2 for these
stencils.  The scaled matrix therefore has ||A||_2 <= 1.
"""
from .problems import (  # noqa: F401
    CSR, Problem, BatchProblem, MultiProblem,
    stencil_2d, stencil_3d, csr_to_dia, normalise, csr_diag,
    poisson_2d, tp2, upwind_2d, upwind_3d,
    problem_poisson2d, problem_convdiff2d, problem_convdiff3d, problem_batched_banded, problem_convdiff2d_multi,
    random_banded_system,
)
