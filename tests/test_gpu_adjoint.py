"""Adjoint gradient of L = ||u - u_obs||^2 through the diffusion solve.

The per-cell kernel is compared with the oracle's gradient formula on the same
(u, lambda, k); the whole autograd chain (forward solve, adjoint solve,
gradient kernel) is compared with central finite differences of the loss,
computed with forward solves only (no oracle involved), and dL/df with the
adjoint itself.
"""
import numpy as np
import pytest

import oracle
from paper_2305_05988_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2305_05988_gb300 as hs  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=torch.float64)


@pytest.mark.parametrize("shape", [(11, 7, 5), (40, 33), (64, 33, 40), (9,)])
def test_gradient_kernel_matches_oracle_formula(shape):
    N = int(np.prod(shape))
    k = np.exp(inputs.normal(2, inputs.STREAM_K, N, 0.5))
    u = inputs.uniform_pm1(41, 1, N)
    lam = inputs.uniform_pm1(42, 1, N)
    g_o = oracle.grad_logk(oracle.Operator(shape, oracle.DIFFUSION, k=k), u, lam)
    kt = dev(k)
    A = hs.Operator.diffusion(shape, kt)
    g = hs.grad_logk(A, dev(u), dev(lam)).cpu().numpy()
    assert np.linalg.norm(g - g_o) <= 1e-13 * np.linalg.norm(g_o)


def _loss(logk, f, u_obs, shape, mixed=False):
    u = hs.diffusion_solve(logk, f, shape, tol=1e-13, mixed=mixed)
    return torch.sum((u - u_obs) ** 2)


@pytest.mark.parametrize("shape,mixed", [((10, 9, 8), False), ((30, 26), False), ((10, 9, 8), True)])
def test_autograd_matches_central_differences(shape, mixed):
    N = int(np.prod(shape))
    logk = dev(inputs.normal(3, inputs.STREAM_K, N, 0.5)).requires_grad_(True)
    f = dev(inputs.uniform_pm1(3, 1, N)).requires_grad_(True)
    k2 = dev(np.exp(inputs.normal(3, inputs.STREAM_K2, N, 0.5)))
    u_obs = hs.cg(hs.Operator.diffusion(shape, k2), f.detach(), tol=1e-13)[0]
    L = _loss(logk, f, u_obs, shape, mixed)
    L.backward()
    g = logk.grad.cpu().numpy()
    gf = f.grad.cpu().numpy()
    rng = np.random.default_rng(7)
    cells = rng.choice(N, size=8, replace=False)
    delta = 1e-4
    fd = []
    with torch.no_grad():
        for c in cells:
            lp = logk.detach().clone()
            lm = logk.detach().clone()
            lp[c] += delta
            lm[c] -= delta
            Lp = _loss(lp, f.detach(), u_obs, shape).item()
            Lm = _loss(lm, f.detach(), u_obs, shape).item()
            fd.append((Lp - Lm) / (2 * delta))
    fd = np.array(fd)
    # central differences carry an O(delta^2) truncation error
    assert np.linalg.norm(g[cells] - fd) <= 1e-6 * np.linalg.norm(fd), (g[cells], fd)
    # dL/df = lambda: u is linear in f, so differences are exact up to rounding
    with torch.no_grad():
        for c in cells[:3]:
            fp = f.detach().clone()
            fm = f.detach().clone()
            fp[c] += 1e-3
            fm[c] -= 1e-3
            d = (_loss(logk.detach(), fp, u_obs, shape).item() - _loss(logk.detach(), fm, u_obs, shape).item()) / 2e-3
            assert abs(d - gf[c]) <= 1e-7 * np.abs(gf).max()


def test_gradient_requires_diffusion_operator():
    A = hs.Operator.laplacian((8, 8))
    u = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        hs.grad_logk(A, u, u)


def test_exp_logk_against_libm_and_in_place():
    # k = exp(log k) on the GPU against numpy's exp: both are within an ulp of
    # the exact exponential, so they differ by at most 2 ulp (4.5e-16 relative)
    N = 100003                        # not a multiple of the block size
    logk = inputs.normal(5, inputs.STREAM_K, N, 1.0) * 3.0
    logk[:4] = [0.0, -700.0, 700.0, 1e-300]
    lt = dev(logk)
    k = hs.exp_logk(lt).cpu().numpy()
    ref = np.exp(logk)
    assert np.all(np.abs(k - ref) <= 4.5e-16 * ref)
    assert k[0] == 1.0 and k[3] == 1.0
    hs.exp_logk(lt, out=lt)           # in place
    assert np.array_equal(lt.cpu().numpy(), k)
    with pytest.raises(TypeError):
        hs.exp_logk(lt.float())


def test_diffusion_solve_forms_k_in_the_library():
    # the differentiable solve's operator uses exp(log k) from hs_exp_logk:
    # its solution equals a solve on that coefficient field
    shape = (20, 17, 9)
    N = int(np.prod(shape))
    logk = dev(inputs.normal(6, inputs.STREAM_K, N, 0.5))
    f = dev(inputs.uniform_pm1(7, 1, N))
    u = hs.diffusion_solve(logk, f, shape, tol=1e-12)
    A = hs.Operator.diffusion(shape, hs.exp_logk(logk))
    u2, info = hs.cg(A, f, tol=1e-12, maxit=100000, history=False)
    assert info.status == "OK"
    assert torch.equal(u, u2)
