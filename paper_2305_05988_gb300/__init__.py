"""GB300-native (sm_103a) structured-grid iterative solvers after arXiv 2305.05988.

Public API: :class:`Operator` (Laplacian / upwind / diffusion stencils),
:func:`jacobi`, :func:`gauss_seidel`, :func:`cg`, :func:`bicgstab`.  The
numerical work runs in libhsolve (hand-written CUDA behind a C ABI,
``include/hsolve.h``); this package only marshals arguments.
"""
from ._lib import HsError  # noqa: F401
from .solvers import (AsyncSolve, Batch, DiffusionSolve, batch_solve, Operator, SolveInfo, bicgstab, cg, cg_nb, diag_wait_timeout,  # noqa: F401
                      diffusion_solve, exp_logk, fp64_rate, gauss_seidel, grad_logk, jacobi, make_opts, solve_mixed)

__all__ = ["HsError", "AsyncSolve", "Batch", "batch_solve", "Operator", "SolveInfo", "jacobi", "gauss_seidel", "cg", "bicgstab", "cg_nb", "solve_mixed", "grad_logk",
           "DiffusionSolve", "diffusion_solve", "make_opts", "diag_wait_timeout", "fp64_rate",
           "exp_logk"]
