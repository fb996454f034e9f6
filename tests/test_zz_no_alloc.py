"""hs_cg_static: the conjugate gradient entry point that allocates nothing.

It serves callers that cannot allocate device memory themselves (for example a
plug-in whose host application owns all GPU memory through its own pool).  The
test calls it through the C ABI twice in a row -- the second call inherits the
first call's leftovers in the shared static scratch -- and checks both results
against hs_cg with a caller-allocated workspace, within the CG parity
tolerance (1e-8 relative), and against the FP64 oracle's CG at the same
iteration count (1e-8 relative), plus the rejection of a problem too large for
the scratch and of a stream that belongs to another device than the current
one (checked only where a second GPU exists).  This file is collected last so that a failure here cannot hide any
other test's result.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2305_05988_gb300 import _lib, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2305_05988_gb300 as hs  # noqa: E402


def _solve_static(A, b, x, tol, maxit):
    lib = _lib.load()
    res = _lib.hs_result()
    hist = np.full(maxit + 1, np.nan)
    st = torch.cuda.current_stream().cuda_stream
    status = lib.hs_cg_static(A._op, _lib.HS_F64, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                              float(tol), int(maxit), None, ctypes.c_void_p(st), ctypes.byref(res),
                              hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return status, res, hist[: res.iters + 1]


@pytest.mark.parametrize("shape", [(37, 19, 11), (128, 128)])
def test_cg_static_matches_cg_on_two_calls_in_a_row(shape):
    A = hs.Operator.laplacian(shape)
    N = A.N
    b = torch.from_numpy(inputs.uniform_pm1(21, 1, N)).cuda()
    x_ref, info = hs.cg(A, b, tol=1e-10, maxit=5000)
    assert info.status == "OK"
    x_o, it_o, st_o, _ = oracle.cg(oracle.Operator(shape), b.cpu().numpy(), tol=0.0, maxit=info.iters)
    assert it_o == info.iters
    for call in range(2):
        x = torch.zeros(N, dtype=torch.float64, device="cuda")
        status, res, hist = _solve_static(A, b, x, 1e-10, 5000)
        assert status == _lib.HS_OK, _lib.load().hs_last_error()
        assert res.status == _lib.HS_OK and res.iters == info.iters
        err = (torch.linalg.norm(x - x_ref) / torch.linalg.norm(x_ref)).item()
        assert err <= 1e-8, (call, err)
        assert np.allclose(hist, info.history, rtol=1e-8, atol=0)
        xh = x.cpu().numpy()
        assert np.linalg.norm(xh - x_o) <= 1e-8 * np.linalg.norm(x_o), call


def test_cg_static_rejects_problems_beyond_its_scratch():
    shape = (256, 256, 64)   # 4 Mi unknowns: 4 FP64 CG vectors need 128 MiB
    A = hs.Operator.laplacian(shape)
    b = torch.ones(A.N, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    status, res, _ = _solve_static(A, b, x, 1e-8, 10)
    assert status == _lib.HS_ERR_INVALID
    msg = _lib.load().hs_last_error().decode()
    assert "static scratch" in msg and str(_lib.HS_STATIC_SCRATCH_BYTES) in msg
    assert torch.count_nonzero(x).item() == 0


def test_cg_static_rejects_a_stream_of_another_device():
    if torch.cuda.device_count() < 2:
        pytest.skip("needs a second GPU")
    A = hs.Operator.laplacian((40, 30))
    b = torch.ones(A.N, dtype=torch.float64, device="cuda:0")
    x = torch.zeros_like(b)
    with torch.cuda.device(1):
        other = torch.cuda.Stream()
    lib = _lib.load()
    res = _lib.hs_result()
    status = lib.hs_cg_static(A._op, _lib.HS_F64, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                              1e-8, 100, None, ctypes.c_void_p(other.cuda_stream), ctypes.byref(res), None)
    assert status == _lib.HS_ERR_INVALID
