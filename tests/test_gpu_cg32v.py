"""The TMA-staged FP32 CG on the 3-D variable-coefficient diffusion operator
(hs_opts.staging = 1: planes staged by TMA, face coefficients formed from k;
csrc/hs_cg32v.cu), as hs_cg with FP32 vectors and as the inner solve of
mixed-precision refinement, against the FP64 oracle.

FP32 tolerances, derived from binary32 arithmetic (unit roundoff u = 6e-8):
the operator forms each face coefficient with a few roundings (harmonic mean
with an approximate division, 2 ulp) and sums 7 terms, so one application of
A to an FP32-representable x is within about 20 u = 1.2e-6 of the FP64
oracle's, relative to ||A x||; each CG iteration adds a similar relative
rounding to the iterate, so iterate k carries about 20 u k relative error on
these well-conditioned early iterations (bar: 1e-5 for k <= 3).  Solutions in
tolerance mode are certified by the oracle's FP64 residual.
"""
import numpy as np
import pytest

import oracle
from paper_2305_05988_gb300 import _lib, inputs
from parity_util import maxrel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2305_05988_gb300 as hs  # noqa: E402

# TMA-eligible grids (n_x a multiple of 4, n_x >= 40): ragged tiles in x
# (44 = 32 + 12) and y, several z chunks, and a larger one
SHAPES = [(64, 33, 40), (44, 21, 13), (40, 10, 3), (96, 50, 70)]


def setup(shape, seed=0, sigma=1.0):
    N = int(np.prod(shape))
    k = np.exp(inputs.normal(seed, inputs.STREAM_K, N, sigma))
    kt = torch.from_numpy(k).cuda()
    return oracle.Operator(shape, oracle.DIFFUSION, k=k), hs.Operator.diffusion(shape, kt), kt


def f32(a):
    return a.astype(np.float32).astype(np.float64)


def staging():
    return _lib.load().hs_last_staging()


@pytest.mark.parametrize("shape", SHAPES)
def test_operator_through_the_initial_residual(shape):
    # maxit = 0 runs the residual pass only: hist[0] = ||b - A x0|| / ||b||
    A_o, A_g, _k = setup(shape)
    b = f32(inputs.uniform_pm1(1, 1, A_o.N))
    x0 = f32(inputs.uniform_pm1(2, 1, A_o.N) * 1e-5)
    bt = torch.from_numpy(b).float().cuda()
    x, info = hs.cg(A_g, bt, torch.from_numpy(x0).float().cuda(), tol=0.0, maxit=0, staging=1)
    assert staging() == 1
    ref = A_o.relres(b, x0)
    assert abs(info.history[0] - ref) <= 2e-6 * ref, (info.history[0], ref)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("k", [1, 2, 3])
def test_early_iterates_against_oracle(shape, k):
    A_o, A_g, _k = setup(shape)
    b = f32(inputs.uniform_pm1(3, 1, A_o.N))
    x_o, _, _, h_o = oracle.cg(A_o, b, tol=0.0, maxit=k)
    x_g, info = hs.cg(A_g, torch.from_numpy(b).float().cuda(), tol=0.0, maxit=k, staging=1)
    assert staging() == 1 and info.iters == k
    xg = x_g.double().cpu().numpy()
    assert np.linalg.norm(xg - x_o) <= 1e-5 * np.linalg.norm(x_o)
    assert maxrel(xg, x_o) <= 1e-5
    assert np.allclose(info.history, h_o, rtol=1e-5, atol=0)


@pytest.mark.parametrize("shape", SHAPES[:3])
def test_tolerance_mode_certified_and_close_to_the_register_engine(shape):
    A_o, A_g, _k = setup(shape)
    b = f32(inputs.uniform_pm1(4, 1, A_o.N))
    bt = torch.from_numpy(b).float().cuda()
    x_t, it_t = hs.cg(A_g, bt, tol=1e-5, maxit=20000, staging=1)
    assert staging() == 1 and it_t.status == "OK"
    x_r, it_r = hs.cg(A_g, bt, tol=1e-5, maxit=20000)
    assert staging() == 0 and it_r.status == "OK"
    # same method, coefficients rounded differently: counts within a few
    assert abs(it_t.iters - it_r.iters) <= max(3, it_r.iters // 50), (it_t.iters, it_r.iters)
    # certified by the oracle's FP64 residual (the recursive FP32 residual
    # drifts from the true one by O(u cond) relative)
    assert A_o.relres(b, x_t.double().cpu().numpy()) <= 2e-5


def test_mixed_refinement_with_tma_inner_solve_certified():
    shape = (64, 48, 40)
    A_o, A_g, _k = setup(shape, seed=5)
    b = inputs.uniform_pm1(6, 1, A_o.N)
    bt = torch.from_numpy(b).cuda()
    x, info = hs.solve_mixed(A_g, bt, tol=1e-10, maxit=30, inner_tol=1e-4, staging=1)
    assert staging() == 1
    assert info.status == "OK" and info.outer >= 2
    assert A_o.relres(b, x.cpu().numpy()) <= 1e-10 * (1 + 1e-3)
    x2, info2 = hs.solve_mixed(A_g, bt, tol=1e-10, maxit=30, inner_tol=1e-4)
    assert staging() == 0 and info2.status == "OK"
    assert A_o.relres(b, x2.cpu().numpy()) <= 1e-10 * (1 + 1e-3)


def test_staging_option_where_it_does_not_apply():
    # n_x not a multiple of 4, a 2-D grid, an FP64 solve: staging = 1 refuses,
    # the default runs the register engine
    A_o, A_g, _k = setup((45, 20, 12))
    bt = torch.from_numpy(f32(inputs.uniform_pm1(7, 1, A_o.N))).float().cuda()
    x, info = hs.cg(A_g, bt, tol=1e-4, maxit=5000)
    assert staging() == 0 and info.status == "OK"
    with pytest.raises(hs.HsError):
        hs.cg(A_g, bt, tol=1e-4, maxit=5000, staging=1)
    with pytest.raises(hs.HsError):
        hs.cg(A_g, bt, tol=1e-4, maxit=5000, staging=2)
    A2_o, A2_g, _k2 = setup((64, 40))
    with pytest.raises(hs.HsError):
        hs.cg(A2_g, torch.ones(A2_o.N, device="cuda"), tol=1e-4, maxit=50, staging=1)
    A3_o, A3_g, _k3 = setup((64, 33, 40))
    with pytest.raises(hs.HsError):
        hs.cg(A3_g, torch.ones(A3_o.N, dtype=torch.float64, device="cuda"), tol=1e-4, maxit=50, staging=1)


def test_zero_rhs_and_nonfinite():
    A_o, A_g, _k = setup((64, 33, 40))
    b = torch.zeros(A_o.N, dtype=torch.float32, device="cuda")
    x, info = hs.cg(A_g, b, torch.ones_like(b), tol=1e-6, maxit=10, staging=1)
    assert staging() == 1 and info.status == "OK" and info.iters == 0
    assert torch.count_nonzero(x).item() == 0
    bn = f32(inputs.uniform_pm1(8, 1, A_o.N))
    bn[1234] = np.nan
    x, info = hs.cg(A_g, torch.from_numpy(bn).float().cuda(), tol=1e-6, maxit=10, staging=1)
    assert info.status == "ERR_NONFINITE"
