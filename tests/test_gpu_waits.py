"""Every kind of device-side wait the kernels use is bounded: run against a
condition that never comes true (a barrier member that is never launched, a
sweep count or progress word that nothing publishes), it gives up after its
limit, the kernel reports ERR_TIMEOUT and the CUDA context stays usable."""
import time

import numpy as np
import pytest

import oracle
from paper_2305_05988_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2305_05988_gb300 as hs  # noqa: E402
from test_gpu_parity import dev, host, rel  # noqa: E402


@pytest.mark.parametrize("kind", ["grid_barrier", "gs_tile", "gs27_ring", "gs27_planes"])
def test_wait_gives_up_and_context_survives(kind):
    t0 = time.time()
    status = hs.diag_wait_timeout(kind, timeout_s=0.05)
    dt = time.time() - t0
    assert status == "ERR_TIMEOUT"
    assert dt < 5.0
    # the context is still usable: a solve right after matches the oracle
    shape = (21, 17, 13)
    A_o = oracle.Operator(shape)
    A_g = hs.Operator.laplacian(shape)
    b = inputs.uniform_pm1(60, 1, A_o.N)
    x_o, _, _, _ = oracle.gauss_seidel(A_o, b, maxit=3)
    x_g, info = hs.gauss_seidel(A_g, dev(b), maxit=3)
    assert info.status == "OK" and rel(host(x_g), x_o) <= 1e-12


def test_wait_limit_is_respected():
    # a longer limit is waited out (not cut short), and still ends
    t0 = time.time()
    assert hs.diag_wait_timeout("gs_tile", timeout_s=0.3) == "ERR_TIMEOUT"
    assert time.time() - t0 >= 0.25
