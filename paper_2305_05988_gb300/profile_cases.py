"""Run one solver case once, for profiling (ncu) and quick timing.

    python -m paper_2305_05988_gb300.profile_cases CASE [N] [ITERS]

CASE picks the kernel: spmv, jacobi, gs, cg, bicgstab, cg_nb (7-point, FP64,
N^3 grid, b ~ U(-1, 1)); jacobi32 (the same in FP32); cg32v (FP32 CG on variable-coefficient diffusion,
log k ~ N(0, 1), stored coefficients), cg32v_tma (the same with TMA-staged
planes); gs2d (Gauss-Seidel on the N^2 Laplacian); hpcg27_spmv, hpcg27_jacobi,
hpcg27_cg, hpcg27_bicgstab, hpcg27_gs (symmetric: the plane-lagged kernel),
hpcg27_gs_hyper (symmetric on the point-hyperplane kernel) and hpcg7_cg (the
HPCG matrices of section 4.1 on 128 x 128 x N, b = A 1).  Each case first runs once to
warm up (CUDA context, workspace), then runs ITERS iterations (sweeps) once
more: profile that second launch (ncu -s <launches of the first run> -c 1).
Prints the wall time of the second run.
"""
from __future__ import annotations

import sys
import time

import numpy as np
import torch

import paper_2305_05988_gb300 as hs
from paper_2305_05988_gb300 import inputs


def main(argv):
    case = argv[1] if len(argv) > 1 else "cg"
    n = int(argv[2]) if len(argv) > 2 else 256
    iters = int(argv[3]) if len(argv) > 3 else 10
    torch.cuda.set_device(0)
    kw = dict(true_residual=False, timeout_s=10.0)
    if case in ("spmv", "jacobi", "gs", "cg", "bicgstab", "cg_nb"):
        shape = (n, n, n)
        b = torch.from_numpy(inputs.rhs_uniform(shape, 0)).cuda()
        A = hs.Operator.upwind(shape, inputs.upwind_beta(shape, 0.5)) if case == "bicgstab" else hs.Operator.laplacian(shape)
        run = {"spmv": lambda: A.spmv(b),
               "jacobi": lambda: hs.jacobi(A, b, maxit=iters, **kw),
               "gs": lambda: hs.gauss_seidel(A, b, maxit=iters, **kw),
               "cg": lambda: hs.cg(A, b, tol=0.0, maxit=iters, history=False, **kw),
               "bicgstab": lambda: hs.bicgstab(A, b, tol=0.0, maxit=iters, history=False, **kw),
               "cg_nb": lambda: hs.cg_nb(A, b, tol=0.0, maxit=iters, history=False, **kw)}[case]
    elif case == "jacobi32":
        shape = (n, n, n)
        b = torch.from_numpy(inputs.rhs_uniform(shape, 0)).float().cuda()
        A = hs.Operator.laplacian(shape)
        run = lambda: hs.jacobi(A, b, maxit=iters, **kw)  # noqa: E731
    elif case in ("cg32v", "cg32v_tma"):
        shape = (n, n, n)
        k = torch.from_numpy(np.exp(inputs.log_k(shape, 1.0, 0))).cuda()
        A = hs.Operator.diffusion(shape, k)
        b = torch.from_numpy(inputs.rhs_uniform(shape, 0)).float().cuda()
        st = 1 if case == "cg32v_tma" else 0
        run = lambda: hs.cg(A, b, tol=0.0, maxit=iters, history=False, staging=st, **kw)  # noqa: E731
    elif case == "gs2d":
        shape = (n, n)
        A = hs.Operator.laplacian(shape)
        b = torch.from_numpy(inputs.rhs_uniform(shape, 0)).cuda()
        run = lambda: hs.gauss_seidel(A, b, maxit=iters, **kw)  # noqa: E731
    elif case.startswith("hpcg"):
        shape = (128, 128, n)
        A = hs.Operator.hpcg(shape, 7 if case.startswith("hpcg7") else 27)
        b = A.spmv(torch.ones(A.N, dtype=torch.float64, device="cuda"))
        which = case.split("_", 1)[1]
        gsk = dict(kw, mode="symmetric", gs_schedule=1 if which == "gs_hyper" else 0)
        run = {"spmv": lambda: A.spmv(b),
               "jacobi": lambda: hs.jacobi(A, b, maxit=iters, **kw),
               "cg": lambda: hs.cg(A, b, tol=0.0, maxit=iters, history=False, **kw),
               "bicgstab": lambda: hs.bicgstab(A, b, tol=0.0, maxit=iters, history=False, **kw),
               "gs": lambda: hs.gauss_seidel(A, b, maxit=iters, **gsk),
               "gs_hyper": lambda: hs.gauss_seidel(A, b, maxit=iters, **gsk)}[which]
    else:
        raise SystemExit("unknown case %r" % case)
    run()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run()
    torch.cuda.synchronize()
    print("%s n=%d iters=%d: %.3f ms" % (case, n, iters, 1e3 * (time.perf_counter() - t0)))


if __name__ == "__main__":
    main(sys.argv)
