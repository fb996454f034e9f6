"""Gauss-Seidel on small 2-D grids by one thread-block cluster (csrc/hs_gs2d.cu,
k_gs2dc: rows split over 8 CTAs, the south / north rows of other CTAs read
through distributed shared memory, a cluster barrier per wavefront step)
against the one-block kernel (max_blocks = 1), the tile schedule
(gs_schedule = 1) and the oracle; gs_schedule = 3 requests the cluster (the
automatic choice takes it for pipelined batches of four or more sweeps).  All three apply the same update to every
node in a lexicographic-compatible order, so the iterates must be bitwise
equal; against the oracle to 1e-12."""
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
    N = int(np.prod(shape))
    if kind == "lap":
        return oracle.Operator(shape), hs.Operator.laplacian(shape), None
    if kind == "up":
        beta = inputs.upwind_beta(shape, 0.5)
        return oracle.Operator(shape, oracle.UPWIND, beta), hs.Operator.upwind(shape, beta), None
    k = np.exp(inputs.normal(0, inputs.STREAM_K, N, 1.0))
    kt = dev(k)
    return oracle.Operator(shape, oracle.DIFFUSION, k=k), hs.Operator.diffusion(shape, kt), kt


# 16 rows: two per CTA; 17: empty CTAs at the top; 23 x 200: ragged rows
SHAPES = [((128, 128), "lap"), ((70, 45), "up"), ((40, 16), "lap"), ((9, 17), "lap"), ((200, 23), "vark"),
          ((33, 64), "vark")]


@pytest.mark.parametrize("shape,kind", SHAPES)
@pytest.mark.parametrize("mode,sweeps", [("forward", 7), ("backward", 3), ("symmetric", 2)])
def test_cluster_equals_one_block_tiles_and_oracle(shape, kind, mode, sweeps):
    A_o, A_g, _k = ops(shape, kind)
    b = inputs.uniform_pm1(81, 1, A_o.N)
    x0 = inputs.uniform_pm1(82, 1, A_o.N)
    x_c, ic = hs.gauss_seidel(A_g, dev(b), dev(x0), maxit=sweeps, mode=mode, gs_schedule=3)
    x_1, i1 = hs.gauss_seidel(A_g, dev(b), dev(x0), maxit=sweeps, mode=mode, max_blocks=1)
    x_t, it = hs.gauss_seidel(A_g, dev(b), dev(x0), maxit=sweeps, mode=mode, gs_schedule=1)
    assert ic.status == "OK" and ic.iters == sweeps
    assert torch.equal(x_c, x_1) and torch.equal(x_c, x_t)
    x_o, _, _, _ = oracle.gauss_seidel(A_o, b, x0, maxit=sweeps, mode=MODES[mode])
    assert maxrel(x_c.cpu().numpy(), x_o) <= 1e-12


def test_cluster_fp32_and_tolerance_mode():
    shape = (96, 80)
    A_o, A_g, _k = ops(shape, "lap")
    b = inputs.uniform_pm1(83, 1, A_o.N)
    x_c, ic = hs.gauss_seidel(A_g, dev(b, torch.float32), maxit=30, gs_schedule=3)
    x_1, i1 = hs.gauss_seidel(A_g, dev(b, torch.float32), maxit=30, max_blocks=1)
    assert torch.equal(x_c, x_1)
    x_c, ic = hs.gauss_seidel(A_g, dev(b), tol=1e-4, maxit=20000, history=True, check_every=3, gs_schedule=3)
    x_1, i1 = hs.gauss_seidel(A_g, dev(b), tol=1e-4, maxit=20000, history=True, check_every=3, max_blocks=1)
    assert ic.status == "OK" and ic.iters == i1.iters
    assert torch.equal(x_c, x_1)
    # the residual norms are reduced in different orders (8 CTAs against one block)
    assert np.allclose(ic.history, i1.history, rtol=1e-12, atol=0, equal_nan=True)


def test_cluster_zero_rhs():
    A_o, A_g, _k = ops((64, 32), "lap")
    b = torch.zeros(A_o.N, dtype=torch.float64, device="cuda")
    x, info = hs.gauss_seidel(A_g, b, torch.ones_like(b), tol=1e-6, maxit=10, gs_schedule=3)
    assert info.status == "OK" and info.iters == 0
    assert torch.count_nonzero(x).item() == 0


def test_cluster_schedule_where_it_does_not_apply():
    A = hs.Operator.laplacian((40, 10))          # fewer than 16 rows
    b = dev(inputs.uniform_pm1(84, 1, 400))
    with pytest.raises(hs.HsError):
        hs.gauss_seidel(A, b, maxit=2, gs_schedule=3)
    A3 = hs.Operator.laplacian((16, 16, 16))
    with pytest.raises(hs.HsError):
        hs.gauss_seidel(A3, dev(inputs.uniform_pm1(85, 1, 4096)), maxit=2, gs_schedule=3)
    A2 = hs.Operator.laplacian((64, 64))
    with pytest.raises(hs.HsError):
        hs.gauss_seidel(A2, dev(inputs.uniform_pm1(86, 1, 4096)), maxit=2, gs_schedule=3, max_blocks=1)
