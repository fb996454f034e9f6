"""Solvers write only inside the workspace they declare: every solver runs on
tiny and ragged grids with a workspace of exactly hs_workspace_size bytes
followed by 4 KB of canary words, and the canary must come back intact (the
stand-in for a memory checker, which is not available on this GPU pool)."""
import ctypes

import numpy as np
import pytest

from paper_2305_05988_gb300 import _lib, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2305_05988_gb300 as hs  # noqa: E402

CANARY = 0x5A3C96E1D2B4F087


def run(A, solver, dtype, b, x, maxit, **kw):
    lib = _lib.load()
    opts = hs.make_opts(**kw)
    need = ctypes.c_size_t()
    dt = _lib.HS_F64 if dtype == torch.float64 else _lib.HS_F32
    assert lib.hs_workspace_size(A._op, solver, dt, ctypes.byref(opts), maxit, ctypes.byref(need)) == 0
    nbytes = (need.value + 255) // 256 * 256
    ws = torch.empty(nbytes + 4096, dtype=torch.uint8, device="cuda")
    tail = ws[nbytes:].view(torch.int64)
    tail.fill_(CANARY)
    res = _lib.hs_result()
    st = torch.cuda.current_stream().cuda_stream
    fn = {_lib.HS_SOLVER_JACOBI: lib.hs_jacobi, _lib.HS_SOLVER_GAUSS_SEIDEL: lib.hs_gauss_seidel,
          _lib.HS_SOLVER_CG: lib.hs_cg, _lib.HS_SOLVER_BICGSTAB: lib.hs_bicgstab,
          _lib.HS_SOLVER_CG_NB: lib.hs_cg_nb}[solver]
    status = fn(A._op, dt, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), 1e-30, maxit,
                ctypes.byref(opts), ctypes.c_void_p(ws.data_ptr()), need.value, ctypes.c_void_p(st),
                ctypes.byref(res), None)
    torch.cuda.synchronize()
    assert status in (_lib.HS_OK, _lib.HS_NOT_CONVERGED, _lib.HS_ERR_BREAKDOWN), status
    assert bool(torch.all(tail == CANARY)), "solver wrote past its workspace"


SHAPES = [(1, 1), (2, 3), (33,), (37, 19, 11), (70, 45), (5, 3, 2), (64, 33, 40)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_solvers_stay_inside_their_workspace(shape, dtype):
    N = int(np.prod(shape))
    k = torch.from_numpy(np.exp(inputs.normal(0, inputs.STREAM_K, N, 1.0))).cuda()
    operators = [("lap", hs.Operator.laplacian(shape)), ("up", hs.Operator.upwind(shape, inputs.upwind_beta(shape, 0.5))),
                 ("vark", hs.Operator.diffusion(shape, k))]
    b = torch.from_numpy(inputs.uniform_pm1(1, 1, N)).to(device="cuda", dtype=dtype)
    for kind, A in operators:
        for solver in (_lib.HS_SOLVER_JACOBI, _lib.HS_SOLVER_GAUSS_SEIDEL, _lib.HS_SOLVER_BICGSTAB):
            run(A, solver, dtype, b, torch.zeros_like(b), 7)
        run(A, _lib.HS_SOLVER_GAUSS_SEIDEL, dtype, b, torch.zeros_like(b), 5, gs_mode="symmetric")
        if kind != "up":
            run(A, _lib.HS_SOLVER_CG, dtype, b, torch.zeros_like(b), 9)
            run(A, _lib.HS_SOLVER_CG_NB, dtype, b, torch.zeros_like(b), 9)
        if kind == "vark" and dtype == torch.float32 and len(shape) == 3 and shape[0] % 4 == 0 and shape[0] >= 40:
            run(A, _lib.HS_SOLVER_CG, dtype, b, torch.zeros_like(b), 9, staging=1)
