"""The pencil schedule of lexicographic Gauss-Seidel (hs_opts.gs_schedule = 2;
the default for batches of four or more sweeps of one direction on 3-D
constant-coefficient operators; csrc/hs_gsp.cu, k_gsp) against the tile
schedule (gs_schedule = 1) and the oracle.

Both schedules apply the same two-part update to every node in an order that
respects the lexicographic dependencies, so their iterates must be bitwise
equal; both must match the oracle's sequential sweep to 1e-12.  The shapes
cover even n_x (pairs loaded as vectors) and odd n_x (a half pair at the end
of every line), grids smaller than one pencil (8 x 4 lines), ragged pencils
in y and z, and few warps for many pencils (max_blocks: each warp then sweeps
several pencils per sweep, in the sweep's direction)."""
import numpy as np
import pytest

import oracle
from paper_2305_05988_gb300 import inputs
from parity_util import maxrel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2305_05988_gb300 as hs  # noqa: E402

MODES = {"forward": oracle.GS_FORWARD, "backward": oracle.GS_BACKWARD, "symmetric": oracle.GS_SYMMETRIC}


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def ops(shape, kind):
    if kind == "lap":
        return oracle.Operator(shape), hs.Operator.laplacian(shape)
    beta = inputs.upwind_beta(shape, 0.5)
    return oracle.Operator(shape, oracle.UPWIND, beta), hs.Operator.upwind(shape, beta)


SHAPES = [(64, 33, 40), (37, 19, 11), (5, 3, 2), (1, 1, 5), (2, 9, 4), (130, 20, 9), (32, 8, 4), (33, 17, 5)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("kind", ["lap", "up"])
@pytest.mark.parametrize("mode,sweeps", [("forward", 5), ("backward", 3), ("symmetric", 2)])
def test_pencils_equal_tiles_and_oracle(shape, kind, mode, sweeps):
    A_o, A_g = ops(shape, kind)
    b = inputs.uniform_pm1(21, 1, A_o.N)
    x0 = inputs.uniform_pm1(22, 1, A_o.N)
    x_p, ip = hs.gauss_seidel(A_g, dev(b), dev(x0), maxit=sweeps, mode=mode, gs_schedule=2)
    x_t, it = hs.gauss_seidel(A_g, dev(b), dev(x0), maxit=sweeps, mode=mode, gs_schedule=1)
    assert ip.status == "OK" and ip.iters == sweeps and it.status == "OK"
    assert torch.equal(x_p, x_t)
    x_o, _, _, _ = oracle.gauss_seidel(A_o, b, x0, maxit=sweeps, mode=MODES[mode])
    assert maxrel(x_p.cpu().numpy(), x_o) <= 1e-12


@pytest.mark.parametrize("blocks", [1, 2, 5])
@pytest.mark.parametrize("mode,sweeps,check_every", [("forward", 7, 1), ("forward", 9, 4), ("symmetric", 3, 1),
                                                     ("symmetric", 4, 2), ("backward", 6, 3)])
def test_pencils_few_warps_and_batches(blocks, mode, sweeps, check_every):
    # 70 x 37 x 41: 5 x 11 = 55 pencils for 4 - 20 warps, tolerance mode with
    # residual checks between batches of sweeps
    shape = (70, 37, 41)
    A_o, A_g = ops(shape, "up")
    b = inputs.uniform_pm1(23, 1, A_o.N)
    x0 = inputs.uniform_pm1(24, 1, A_o.N)
    kw = dict(maxit=sweeps, mode=mode, tol=1e-300, check_every=check_every, max_blocks=blocks)
    x_p, ip = hs.gauss_seidel(A_g, dev(b), dev(x0), gs_schedule=2, history=True, **kw)
    x_t, it = hs.gauss_seidel(A_g, dev(b), dev(x0), gs_schedule=1, history=True, **kw)
    assert ip.iters == sweeps and ip.status == "NOT_CONVERGED", ip
    assert torch.equal(x_p, x_t)
    # the residual norms are reduced over launch shapes of different sizes
    # (the order of the deterministic reduction follows the grid), so they
    # agree to rounding, not bitwise
    assert np.allclose(ip.history, it.history, rtol=1e-13, atol=0, equal_nan=True)
    x_o, _, _, _ = oracle.gauss_seidel(A_o, b, x0, maxit=sweeps, mode=MODES[mode])
    assert maxrel(x_p.cpu().numpy(), x_o) <= 1e-12


def test_pencils_fp32_and_tolerance_mode():
    shape = (48, 26, 18)
    A_o, A_g = ops(shape, "lap")
    b = inputs.uniform_pm1(25, 1, A_o.N)
    bt = dev(b, torch.float32)
    x_p, ip = hs.gauss_seidel(A_g, bt, maxit=40, gs_schedule=2)
    x_t, it = hs.gauss_seidel(A_g, bt, maxit=40, gs_schedule=1)
    assert torch.equal(x_p, x_t)
    x_p, ip = hs.gauss_seidel(A_g, dev(b), tol=1e-6, maxit=5000, gs_schedule=2, history=True)
    x_t, it = hs.gauss_seidel(A_g, dev(b), tol=1e-6, maxit=5000, gs_schedule=1, history=True)
    assert ip.status == "OK" and ip.iters == it.iters
    assert torch.equal(x_p, x_t)
    x_o, it_o, st_o, _ = oracle.gauss_seidel(A_o, b, maxit=5000, tol=1e-6)
    assert ip.iters == it_o


def test_pencil_schedule_only_for_3d_constant_coefficients():
    k = dev(np.exp(inputs.normal(0, inputs.STREAM_K, 20 * 9 * 6, 0.5)))
    A_v = hs.Operator.diffusion((20, 9, 6), k)
    b = dev(inputs.uniform_pm1(26, 1, 20 * 9 * 6))
    with pytest.raises(hs.HsError):
        hs.gauss_seidel(A_v, b, maxit=2, gs_schedule=2)
    x, info = hs.gauss_seidel(A_v, b, maxit=2)          # the tile schedule
    assert info.status == "OK"
    A2 = hs.Operator.laplacian((40, 30))
    with pytest.raises(hs.HsError):
        hs.gauss_seidel(A2, dev(inputs.uniform_pm1(27, 1, 1200)), maxit=2, gs_schedule=2)
    with pytest.raises(hs.HsError):
        hs.gauss_seidel(A2, dev(inputs.uniform_pm1(27, 1, 1200)), maxit=2, gs_schedule=4)
