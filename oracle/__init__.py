"""CPU oracle for the p-BiCGStab hot path (arXiv 1809.01948).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this package.  The
product path (the CUDA library and its Python binding) never calls it, and it
shares no code with the CUDA path; inputs come from the separate
``testproblems`` module.

Plain, slow, obviously-correct numpy/scipy code in FP64 (plus a mixed
FP32/FP64 emulation mode), following the paper's algorithms step by step:

* ``bicgstab``      -- Algorithm 1 (classic preconditioned BiCGStab).
* ``pbicgstab``     -- Algorithm 2 (preconditioned pipelined BiCGStab) with the
                       residual replacement step of Eq. (rr), periodic and
                       automated (Eq. DDr_bound / criterion) policies.
* ``diagnostics``   -- measured local rounding errors of Eq. (auxrec), the gaps
                       of Eq. (DsDwDz)/(res_gap), the error bounds
                       Eq. (errbounds1)-(errbounds4) and the gap bound f^r.
* ``adjoint``       -- dense and sparse adjoint gradients for the
                       differentiable solve (standard linear algebra, not in
                       the paper).

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against library routines (scipy's BiCGStab, LAPACK dense solves), closed forms
and the paper's invariants, except the mixed-precision emulation, which is
"parity partially pinned" (see ``pbicgstab`` docstring).
"""
from .precond import Identity, Jacobi, Neumann, make_precond  # noqa: F401
from .krylov import bicgstab, pbicgstab, SolveResult, Status  # noqa: F401
from .krylov import spmv  # noqa: F401
from . import diagnostics, adjoint  # noqa: F401
