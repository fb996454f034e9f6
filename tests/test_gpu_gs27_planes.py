"""The plane-lagged lexicographic Gauss-Seidel for the HPCG 27-point operator
(csrc/hs_gs27.cu, k_gs27p; hs_opts.gs_schedule = 2): whole z planes per block
in shared memory, in-plane steps i + 2j, each plane four steps behind the one
below it.  Against the hyperplane kernel (gs_schedule = 1, one grid-wide step
per point hyperplane i + 2j + 4k): both apply the same update to every node in
an order compatible with the lexicographic one, so the iterates, residual
histories and iteration counts must be bitwise equal; against the oracle to
1e-12 (FP64)."""
import time

import numpy as np
import pytest

import oracle
from paper_2305_05988_gb300 import inputs
from parity_util import maxrel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2305_05988_gb300 as hs  # noqa: E402
from paper_2305_05988_gb300._lib import HS_ERR_INVALID  # noqa: E402

MODES = {"forward": oracle.GS_FORWARD, "backward": oracle.GS_BACKWARD, "symmetric": oracle.GS_SYMMETRIC}
# ragged planes, one-node lines and planes, more blocks than planes
SHAPES = [(37, 19, 11), (5, 4, 3), (1, 9, 7), (8, 1, 5), (6, 5, 1), (1, 1, 1), (2, 1, 9), (33, 8, 70),
          (9, 13, 2)]


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def both(A_g, b, x0, **kw):
    xs = [hs.gauss_seidel(A_g, b, x0.clone(), gs_schedule=s, **kw) for s in (1, 2)]
    return xs[0], xs[1]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("mode", ["forward", "backward", "symmetric"])
def test_planes_equal_hyperplanes_and_oracle(shape, mode):
    A_o = oracle.Operator(shape, oracle.HPCG27)
    A_g = hs.Operator.hpcg(shape, 27)
    b = inputs.uniform_pm1(71, 1, A_o.N)
    x0 = inputs.uniform_pm1(72, 1, A_o.N)
    for k in (1, 2, 5):
        (xh, ih), (xp, ip) = both(A_g, dev(b), dev(x0), maxit=k, mode=mode)
        assert ih.iters == ip.iters == k
        assert np.array_equal(host(xh), host(xp)), (shape, mode, k)
        x_o, _, _, _ = oracle.gauss_seidel(A_o, b, x0, maxit=k, mode=MODES[mode])
        assert maxrel(host(xp), x_o) <= 1e-12
    bf, xf0 = dev(b, torch.float32), dev(x0, torch.float32)
    (xh, _), (xp, _) = both(A_g, bf, xf0, maxit=3, mode=mode)
    assert torch.equal(xh, xp)


@pytest.mark.parametrize("blocks", [1, 2, 3, 7])
def test_planes_few_blocks(blocks):
    # plane k belongs to block k mod G: with few blocks each owns several
    # planes and waits on its own earlier planes' neighbours
    shape = (9, 6, 23)
    A_o = oracle.Operator(shape, oracle.HPCG27)
    A_g = hs.Operator.hpcg(shape, 27)
    b = inputs.uniform_pm1(73, 1, A_o.N)
    x0 = inputs.uniform_pm1(74, 1, A_o.N)
    for mode in ("forward", "backward", "symmetric"):
        (xh, _), (xp, ip) = both(A_g, dev(b), dev(x0), maxit=4, mode=mode, max_blocks=blocks)
        assert ip.iters == 4 and np.array_equal(host(xh), host(xp)), (mode, blocks)
        # residual checks every 2 sweeps: batches of two, sweep counts go on
        (xh, ih), (xp, ip) = both(A_g, dev(b), dev(x0), maxit=5, mode=mode, max_blocks=blocks, tol=1e-300,
                                  check_every=2, history=True)
        assert ih.iters == ip.iters == 5 and np.array_equal(host(xh), host(xp)), (mode, blocks)
        assert np.allclose(np.asarray(ih.history), np.asarray(ip.history), rtol=1e-13, atol=0, equal_nan=True)


@pytest.mark.parametrize("mode", ["forward", "symmetric"])
def test_planes_to_tolerance(mode):
    shape = (24, 20, 18)
    A_o = oracle.Operator(shape, oracle.HPCG27)
    A_g = hs.Operator.hpcg(shape, 27)
    b = A_o.spmv(np.ones(A_o.N))
    tol = 1e-6 / np.linalg.norm(b)
    (xh, ih), (xp, ip) = both(A_g, dev(b), torch.zeros(A_o.N, dtype=torch.float64, device="cuda"), tol=tol,
                              maxit=2000, mode=mode, check_every=1, history=True)
    assert ih.status == ip.status == "OK" and ih.iters == ip.iters
    assert np.array_equal(host(xh), host(xp))
    # the residual's grid reduction is summed in an order set by the grid
    # (one block per SM against one per plane here), hence not bitwise
    assert np.allclose(np.asarray(ih.history), np.asarray(ip.history), rtol=1e-13, atol=0)
    assert np.linalg.norm(b - A_o.spmv(host(xp))) <= 1e-6 * (1 + 1e-3)


def test_planes_option_validation():
    A_g = hs.Operator.hpcg((256, 256, 3), 27)   # a 512 KB FP64 plane
    b = torch.ones(256 * 256 * 3, dtype=torch.float64, device="cuda")
    with pytest.raises(hs.HsError) as e:
        hs.gauss_seidel(A_g, b, maxit=1, gs_schedule=2)
    assert e.value.status == HS_ERR_INVALID
    with pytest.raises(hs.HsError) as e:
        hs.gauss_seidel(A_g, b, maxit=1, gs_schedule=3)
    assert e.value.status == HS_ERR_INVALID
    # the automatic choice falls back to the hyperplane kernel
    x, info = hs.gauss_seidel(A_g, b, maxit=1, mode="symmetric")
    assert info.iters == 1
    x1, _ = hs.gauss_seidel(A_g, b, maxit=1, mode="symmetric", gs_schedule=1)
    assert torch.equal(x, x1)
    # an FP32 plane of 128 x 256 nodes (128 KB) fits
    A32 = hs.Operator.hpcg((128, 256, 5), 27)
    b32 = torch.ones(128 * 256 * 5, dtype=torch.float32, device="cuda")
    xa, _ = hs.gauss_seidel(A32, b32, maxit=2, gs_schedule=2)
    xb, _ = hs.gauss_seidel(A32, b32, maxit=2, gs_schedule=1)
    assert torch.equal(xa, xb)


def test_planes_wide_steps():
    # 100 nodes per in-plane step at the widest: 200 of the 224 compute lanes
    shape = (250, 100, 4)
    A_g = hs.Operator.hpcg(shape, 27)
    N = int(np.prod(shape))
    b = dev(inputs.uniform_pm1(77, 1, N))
    x0 = dev(inputs.uniform_pm1(78, 1, N))
    for mode in ("forward", "symmetric"):
        (xh, _), (xp, _) = both(A_g, b, x0, maxit=2, mode=mode)
        assert torch.equal(xh, xp), mode


def test_planes_hpcg_plane_size_symmetric():
    # the paper's plane size (128 x 128) over 96 planes; prints the time per
    # symmetric iteration of both kernels
    shape = (128, 128, 96)
    N = int(np.prod(shape))
    A_g = hs.Operator.hpcg(shape, 27)
    b = dev(inputs.uniform_pm1(75, 1, N))
    x0 = dev(inputs.uniform_pm1(76, 1, N))
    out = {}
    for s in (1, 2):
        hs.gauss_seidel(A_g, b, x0.clone(), maxit=1, mode="symmetric", gs_schedule=s)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, info = hs.gauss_seidel(A_g, b, x0.clone(), maxit=2, mode="symmetric", gs_schedule=s)
        torch.cuda.synchronize()
        out[s] = (x, (time.perf_counter() - t0) / 2)
    print("128x128x96 symmetric GS per iteration: hyperplanes %.2f ms, planes %.2f ms"
          % (out[1][1] * 1e3, out[2][1] * 1e3))
    assert torch.equal(out[1][0], out[2][0])
