"""The asynchronous solver forms (hs_jacobi_async, hs_gauss_seidel_async,
hs_cg_async, hs_bicgstab_async; Python AsyncSolve): the outcome and history
written into device memory by the library, nothing on the host waiting, so a
solve can be captured in a CUDA graph and replayed.

Each form runs exactly the synchronous solver's kernels, so its iterate,
iteration count, status and residuals must equal the synchronous call's
bitwise; a graph replayed with new right-hand sides must give what a fresh
synchronous solve gives, and the synchronous solve is checked against the
oracle in the parity tests."""
import numpy as np
import pytest

from paper_2305_05988_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2305_05988_gb300 as hs  # noqa: E402


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def op(shape, kind):
    if kind == "lap":
        return hs.Operator.laplacian(shape)
    return hs.Operator.upwind(shape, inputs.upwind_beta(shape, 0.5))


SYNC = {"jacobi": hs.jacobi, "gauss_seidel": hs.gauss_seidel, "cg": hs.cg, "bicgstab": hs.bicgstab}

CASES = [
    ("jacobi", "lap", (37, 19, 11), dict(tol=0.0, maxit=40)),
    ("jacobi", "up", (40, 30), dict(tol=1e-4, maxit=5000, history=True)),
    ("gauss_seidel", "lap", (64, 33, 40), dict(tol=0.0, maxit=9, gs_schedule=2)),       # pencils
    ("gauss_seidel", "lap", (64, 33, 40), dict(tol=0.0, maxit=9)),                      # tiles
    ("gauss_seidel", "up", (37, 19, 11), dict(tol=0.0, maxit=3, mode="symmetric")),     # tiles
    ("gauss_seidel", "lap", (45, 38), dict(tol=1e-3, maxit=2000, history=True)),        # one block
    ("gauss_seidel", "lap", (64, 48), dict(tol=0.0, maxit=6)),                          # one cluster
    ("cg", "lap", (64, 33, 40), dict(tol=1e-10, maxit=5000, history=True)),
    ("cg", "lap", (70, 45), dict(tol=1e-10, maxit=5000, history=True)),
    ("bicgstab", "up", (64, 33, 40), dict(tol=1e-10, maxit=5000, history=True)),
]


@pytest.mark.parametrize("solver,kind,shape,kw", CASES)
def test_async_form_equals_synchronous_call(solver, kind, shape, kw):
    A = op(shape, kind)
    N = int(np.prod(shape))
    b = dev(inputs.uniform_pm1(41, 1, N))
    x0 = dev(inputs.uniform_pm1(42, 1, N) * 0.1)
    kw = dict(kw)
    hist = kw.pop("history", False)
    x_s, i_s = SYNC[solver](A, b, x0, history=hist, **kw)
    x_a = x0.clone()
    job = hs.AsyncSolve(solver, A, b, x_a, history=hist, **kw)
    job.launch()
    i_a = job.result()
    assert torch.equal(x_a, x_s)
    assert (i_a.iters, i_a.status, i_a.restarts) == (i_s.iters, i_s.status, i_s.restarts)
    assert i_a.rel_res == i_s.rel_res and i_a.true_rel_res == i_s.true_rel_res
    if hist and i_s.history is not None:
        assert np.array_equal(i_a.history, i_s.history, equal_nan=True)


@pytest.mark.parametrize("solver,kind,shape,kw", [
    ("cg", "lap", (64, 33, 40), dict(tol=1e-9, maxit=5000)),
    ("bicgstab", "up", (48, 40, 36), dict(tol=1e-9, maxit=5000)),
    ("gauss_seidel", "lap", (64, 33, 40), dict(tol=0.0, maxit=6)),
    ("gauss_seidel", "lap", (64, 33, 40), dict(tol=0.0, maxit=6, gs_schedule=2)),
    ("gauss_seidel", "up", (37, 19, 11), dict(tol=0.0, maxit=2, mode="symmetric")),
    ("gauss_seidel", "lap", (64, 48), dict(tol=0.0, maxit=6)),
    ("jacobi", "lap", (64, 33, 40), dict(tol=0.0, maxit=30)),
])
def test_async_solve_captured_in_a_cuda_graph(solver, kind, shape, kw):
    A = op(shape, kind)
    N = int(np.prod(shape))
    b = torch.zeros(N, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    job = hs.AsyncSolve(solver, A, b, x, **kw)
    b.copy_(dev(inputs.uniform_pm1(50, 1, N)))
    job.launch()                                   # outside capture first
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        job.launch()
    for seed in (51, 52, 53):
        bn = dev(inputs.uniform_pm1(seed, 1, N))
        b.copy_(bn)
        x.zero_()
        g.replay()
        torch.cuda.synchronize()
        x_s, i_s = SYNC[solver](A, bn, **kw)
        i_g = job.result()
        assert torch.equal(x, x_s), seed
        assert (i_g.iters, i_g.status) == (i_s.iters, i_s.status), seed
        assert i_g.true_rel_res == i_s.true_rel_res


def test_async_form_rejects_what_it_cannot_do():
    A = op((20, 17, 9), "up")
    N = 20 * 17 * 9
    b = dev(inputs.uniform_pm1(60, 1, N))
    x = torch.zeros_like(b)
    with pytest.raises(ValueError):
        hs.AsyncSolve("solve_mixed", A, b, x)
    with pytest.raises(hs.HsError):                  # CG on a nonsymmetric operator
        hs.AsyncSolve("cg", A, b, x).launch()
    with pytest.raises(hs.HsError):                  # negative tolerance
        hs.AsyncSolve("bicgstab", A, b, x, tol=-1.0).launch()
    job = hs.AsyncSolve("bicgstab", A, b, x, tol=1e-8)
    alpha = np.zeros(10001)
    job.opts.alpha_trace = alpha.ctypes.data_as(__import__("ctypes").POINTER(__import__("ctypes").c_double))
    with pytest.raises(hs.HsError):                  # the host-side trace is not asynchronous
        job.launch()
