"""Temporally blocked Jacobi (several sweeps per pass over the grid): the
iterates must be bitwise those of one sweep per pass (same arithmetic per
node), and match the FP64 oracle to 1e-12 after k sweeps."""
import numpy as np
import pytest

import oracle
from paper_2305_05988_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2305_05988_gb300 as hs  # noqa: E402
from test_gpu_parity import dev, host, rel  # noqa: E402

CASES = [((37, 19, 11), "lap"), ((64, 33, 40), "lap"), ((70, 9, 130), "lap"), ((40, 24, 33), "hpcg7"),
         ((3, 2, 5), "lap")]


def gpu_op(shape, kind):
    return hs.Operator.laplacian(shape) if kind == "lap" else hs.Operator.hpcg(shape, 7)


def ora_op(shape, kind):
    return oracle.Operator(shape) if kind == "lap" else oracle.Operator(shape, oracle.HPCG7)


@pytest.mark.parametrize("shape,kind", CASES)
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_blocked_sweeps_bitwise_equal_single_sweeps(shape, kind, dtype):
    A = gpu_op(shape, kind)
    N = int(np.prod(shape))
    b = dev(inputs.uniform_pm1(61, 1, N), dtype)
    x0 = dev(inputs.uniform_pm1(62, 1, N), dtype)
    for sweeps in (1, 2, 7, 10):
        ref, _ = hs.jacobi(A, b, x0.clone(), maxit=sweeps)
        for spp in (2, 3, 4):
            x, info = hs.jacobi(A, b, x0.clone(), maxit=sweeps, sweeps_per_pass=spp)
            assert info.iters == sweeps and info.status == "OK"
            assert torch.equal(x, ref), (sweeps, spp)


@pytest.mark.parametrize("shape,kind", CASES[:4])
def test_blocked_sweeps_match_oracle(shape, kind):
    A_o, A_g = ora_op(shape, kind), gpu_op(shape, kind)
    b = inputs.uniform_pm1(63, 1, A_o.N)
    x0 = inputs.uniform_pm1(64, 1, A_o.N)
    x_o, _, _, _ = oracle.jacobi(A_o, b, x0, maxit=9)
    x_g, info = hs.jacobi(A_g, dev(b), dev(x0), maxit=9, sweeps_per_pass=3)
    assert rel(host(x_g), x_o) <= 1e-12


def test_blocked_sweeps_fall_back_where_not_applicable():
    # tolerance mode, 2-D and the upwind operator run one sweep per pass
    shape = (30, 20, 10)
    A = hs.Operator.laplacian(shape)
    b = dev(inputs.uniform_pm1(65, 1, 6000))
    x1, i1 = hs.jacobi(A, b, tol=1e-3, maxit=500)
    x2, i2 = hs.jacobi(A, b, tol=1e-3, maxit=500, sweeps_per_pass=2)
    assert i1.iters == i2.iters and torch.equal(x1, x2)
    A2 = hs.Operator.laplacian((50, 40))
    b2 = dev(inputs.uniform_pm1(66, 1, 2000))
    assert torch.equal(hs.jacobi(A2, b2, maxit=5)[0], hs.jacobi(A2, b2, maxit=5, sweeps_per_pass=2)[0])
