"""Tiny and ragged parity cases run against the debug build of libhsolve
(HSOLVE_DEBUG=1: every global index the tile engines form is checked; a bad
one is reported as ERR_BOUNDS instead of being used).  Run by
tests/test_gpu_debug_build.py in a child process with HSOLVE_DEBUG=1; exits
non-zero on the first failure.  Not collected by pytest (no test_ prefix)."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import torch  # noqa: E402

import oracle  # noqa: E402
import paper_2305_05988_gb300 as hs  # noqa: E402
from paper_2305_05988_gb300 import _build, _lib, inputs  # noqa: E402
from parity_util import maxrel  # noqa: E402

# a fixed-count Krylov run ends OK (converged exactly), NOT_CONVERGED (ran
# maxit) or, on a 1-node grid, in a breakdown; ERR_BOUNDS would be a fired check
RUN_OK = ("OK", "NOT_CONVERGED", "ERR_BREAKDOWN")
SHAPES = [(1, 1), (2, 3), (5, 4), (3, 4, 5), (33,), (37, 19, 11), (70, 45), (31, 17, 9), (64, 33, 40), (5, 3, 2)]


def ops(shape, kind):
    N = int(np.prod(shape))
    if kind == "lap":
        return oracle.Operator(shape), hs.Operator.laplacian(shape), None
    if kind == "up":
        beta = inputs.upwind_beta(shape, 0.5)
        return oracle.Operator(shape, oracle.UPWIND, beta), hs.Operator.upwind(shape, beta), None
    k = np.exp(inputs.normal(0, inputs.STREAM_K, N, 1.0))
    kt = torch.from_numpy(k).cuda()
    return oracle.Operator(shape, oracle.DIFFUSION, k=k), hs.Operator.diffusion(shape, kt), kt


def dev(a, dt=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)


def main():
    assert _build.DEBUG and "_build_debug" in _lib.lib_path(), "not the debug build"
    n = 0
    for shape in SHAPES:
        for kind in ("lap", "up", "vark"):
            A_o, A_g, _k = ops(shape, kind)
            b = inputs.uniform_pm1(1, 1, A_o.N)
            x0 = inputs.uniform_pm1(2, 1, A_o.N)
            y = A_g.spmv(dev(x0)).cpu().numpy()
            assert maxrel(y, A_o.spmv(x0)) <= 1e-13, (shape, kind)
            r = A_g.residual(dev(b), dev(x0)).cpu().numpy()
            assert maxrel(r, b - A_o.spmv(x0)) <= 1e-13, (shape, kind)
            xj, info = hs.jacobi(A_g, dev(b), dev(x0), maxit=5)
            assert info.status == "OK" and maxrel(xj.cpu().numpy(), oracle.jacobi(A_o, b, x0, maxit=5)[0]) <= 1e-12
            for mode, m in (("forward", oracle.GS_FORWARD), ("symmetric", oracle.GS_SYMMETRIC)):
                xg, info = hs.gauss_seidel(A_g, dev(b), dev(x0), maxit=3, mode=mode)
                ref = oracle.gauss_seidel(A_o, b, x0, maxit=3, mode=m)[0]
                assert info.status == "OK" and maxrel(xg.cpu().numpy(), ref) <= 1e-12, (shape, kind, mode)
            if kind != "up":
                xc, info = hs.cg(A_g, dev(b), tol=0.0, maxit=4)
                assert info.status in RUN_OK, (shape, kind, info.status)
                assert maxrel(xc.cpu().numpy(), oracle.cg(A_o, b, tol=0.0, maxit=info.iters)[0]) <= 1e-9
                xn, info = hs.cg_nb(A_g, dev(b), tol=0.0, maxit=4)
                assert info.status in RUN_OK, (shape, kind, info.status)
            xb, info = hs.bicgstab(A_g, dev(b), tol=0.0, maxit=3)
            assert info.status in RUN_OK, (shape, kind, info.status)
            n += 1
    # the TMA-staged FP32 CG (n_x a multiple of 4, n_x >= 40) on ragged tiles
    for shape in ((44, 21, 13), (40, 10, 3), (64, 33, 40)):
        A_o, A_g, _k = ops(shape, "vark")
        b = inputs.uniform_pm1(3, 1, A_o.N).astype(np.float32)
        x, info = hs.cg(A_g, dev(b, torch.float32), tol=0.0, maxit=3, staging=1)
        assert info.status in RUN_OK and _lib.load().hs_last_staging() == 1, (shape, info.status)
        n += 1
    print("debug build: %d cases, no bounds check fired" % n)


if __name__ == "__main__":
    main()
