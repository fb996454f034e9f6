"""Mixed-precision iterative refinement (FP32 inner solves, FP64 residual and
update) against the FP64 oracle.

Every result is certified by the oracle's own FP64 SpMV (true relative
residual <= tol) and its error against the oracle's FP64 solution is reported
and bounded by the forward-error bound kappa_2(A) * (residual of both
solutions), with kappa_2 from a dense SVD on these small grids.
"""
import numpy as np
import pytest

import oracle
from paper_2305_05988_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2305_05988_gb300 as hs  # noqa: E402


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def ops(shape, kind, sigma=1.0):
    N = int(np.prod(shape))
    if kind == "lap":
        return oracle.Operator(shape), hs.Operator.laplacian(shape), None
    if kind == "up":
        beta = inputs.upwind_beta(shape, 0.5)
        return oracle.Operator(shape, oracle.UPWIND, beta), hs.Operator.upwind(shape, beta), None
    k = np.exp(inputs.normal(0, inputs.STREAM_K, N, sigma))
    kt = dev(k)
    return oracle.Operator(shape, oracle.DIFFUSION, k=k), hs.Operator.diffusion(shape, kt), kt


@pytest.mark.parametrize("shape,kind,inner", [((20, 14, 9), "vark", "cg"), ((45, 38), "vark", "cg"),
                                              ((33, 27), "lap", "cg"), ((24, 20, 8), "up", "bicgstab"),
                                              ((45, 38), "vark", "bicgstab")])
def test_mixed_reaches_fp64_accuracy(shape, kind, inner):
    A_o, A_g, _k = ops(shape, kind)
    N = A_o.N
    b = inputs.uniform_pm1(31, 1, N)
    tol = 1e-10
    x, info = hs.solve_mixed(A_g, dev(b), tol=tol, maxit=30, inner_solver=inner)
    assert info.status == "OK", info
    xh = x.cpu().numpy()
    true_rel = A_o.relres(b, xh)
    assert true_rel <= tol * (1 + 1e-3)
    assert abs(true_rel - info.true_rel_res) <= 1e-3 * tol + 1e-16
    assert info.history[-1] <= tol and info.outer >= 1 and info.inner_iters > 0
    # error against the oracle's FP64 solution
    M = A_o.dense(maxN=4096)
    x_ref = np.linalg.solve(M, b)
    kappa = np.linalg.cond(M)
    err = np.linalg.norm(xh - x_ref) / np.linalg.norm(x_ref)
    assert err <= kappa * 2 * tol, (err, kappa)


def test_mixed_matches_oracle_cg_solution():
    shape = (37, 19, 11)
    A_o, A_g, _k = ops(shape, "vark")
    b = inputs.uniform_pm1(32, 1, A_o.N)
    x_o, it_o, st_o, _ = oracle.cg(A_o, b, tol=1e-12, maxit=20000)
    x, info = hs.solve_mixed(A_g, dev(b), tol=1e-12, maxit=30)
    assert info.status == "OK"
    err = np.linalg.norm(x.cpu().numpy() - x_o) / np.linalg.norm(x_o)
    assert err <= 1e-8, err


def test_fp32_dots_are_fp64_accumulated():
    # hist[0] of an FP32 CG solve is sqrt(r.r / b.b) with r = b - A x0 in FP32;
    # with both dots accumulated in FP64 from exactly widened FP32 values it
    # matches the FP64 sums of the same FP32 data to ~1e-15, far below what an
    # FP32 accumulation over 7733 terms could give.
    shape = (37, 19, 11)
    A_g = hs.Operator.laplacian(shape)
    N = A_g.N
    b = dev(inputs.uniform_pm1(33, 1, N), torch.float32)
    x0 = dev(inputs.uniform_pm1(34, 1, N) * 1e-4, torch.float32)
    r = A_g.residual(b, x0).cpu().numpy().astype(np.float64)
    bb = b.cpu().numpy().astype(np.float64)
    ref = np.sqrt(np.dot(r, r) / np.dot(bb, bb))
    _, info = hs.cg(A_g, b, x0, tol=1e-3, maxit=50)
    assert abs(info.history[0] - ref) <= 1e-13 * ref


def test_mixed_zero_rhs_and_errors():
    A_o, A_g, _k = ops((20, 14, 9), "vark")
    b = torch.zeros(A_o.N, dtype=torch.float64, device="cuda")
    x, info = hs.solve_mixed(A_g, b, x0=torch.ones_like(b), tol=1e-10)
    assert info.status == "OK" and info.outer == 0 and torch.count_nonzero(x).item() == 0
    bn = inputs.uniform_pm1(35, 1, A_o.N)
    bn[3] = np.inf
    x, info = hs.solve_mixed(A_g, dev(bn), tol=1e-10)
    assert info.status == "ERR_NONFINITE"
    with pytest.raises(TypeError):
        hs.solve_mixed(A_g, b.float())
    U_o, U_g, _ = ops((20, 14), "up")
    with pytest.raises(hs.solvers._lib.HsError):
        hs.solve_mixed(U_g, dev(inputs.uniform_pm1(36, 1, U_o.N)), inner_solver="cg")


@pytest.mark.parametrize("inner", ["cg", "bicgstab"])
def test_last_step_stops_its_inner_solve_at_what_tol_needs(inner):
    # inner_fixed_tol = 0 (default): a refinement step with FP64 relative
    # residual rel runs its inner solve to max(inner_tol, 0.5 tol / rel) only.
    # Every step before the first one where that bound exceeds inner_tol is
    # the same computation in both modes (bitwise equal histories); the
    # adaptive run takes no more inner iterations, and both are certified.
    shape = (64, 48, 40)
    A_o, A_g, _k = ops(shape, "vark")
    b = inputs.uniform_pm1(37, 1, A_o.N)
    tol, itol = 1e-10, 1e-4
    xf, f = hs.solve_mixed(A_g, dev(b), tol=tol, maxit=30, inner_tol=itol, inner_solver=inner, inner_fixed_tol=1)
    xa, a = hs.solve_mixed(A_g, dev(b), tol=tol, maxit=30, inner_tol=itol, inner_solver=inner)
    assert f.status == "OK" and a.status == "OK"
    for x in (xf, xa):
        assert A_o.relres(b, x.cpu().numpy()) <= tol * (1 + 1e-3)
    k = next(k for k in range(len(f.history)) if 0.5 * tol / f.history[k] > itol)
    assert np.array_equal(a.history[:k + 1], f.history[:k + 1]), (a.history, f.history)
    assert a.inner_iters <= f.inner_iters, (a.inner_iters, f.inner_iters)
    print("inner iterations: fixed %d (%d steps), adaptive %d (%d steps)" % (f.inner_iters, f.outer, a.inner_iters,
                                                                            a.outer))
