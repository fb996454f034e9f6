"""The paper's proposed Krylov variants on the GPU, against the FP64 oracle:
CG-NB (Algorithm 1; one fused pass and one grid reduction per iteration) and
BiCGStab in Algorithm 2's statement order (BiCGStab-B1, paper_order=True).

Tolerances: iterates at equal iteration counts within 1e-8 (relative; the
GPU expands CG-NB's denominator (A p).p into r.A r - beta r.r / alpha, which
rounds differently from the oracle's direct dot); in tolerance mode counts
within +-2 of the oracle's and the oracle certifies the true residual.
"""
import numpy as np
import pytest

import oracle
from paper_2305_05988_gb300 import inputs
from parity_util import iterate_bar, oracle_window, oracle_xdev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2305_05988_gb300 as hs  # noqa: E402
from test_gpu_parity import dev, host, make_ops, rel  # noqa: E402

NB_CASES = [((128, 128), "lap"), ((70, 45), "vark"), ((37, 19, 11), "lap"), ((64, 33, 40), "lap"),
            ((30, 22, 17), "vark"), ((33,), "lap")]


@pytest.mark.parametrize("shape,kind", NB_CASES)
def test_cg_nb_iterates_match_oracle(shape, kind):
    A_o, A_g, _k = make_ops(shape, kind)
    b = inputs.uniform_pm1(31, 1, A_o.N)
    for k in (1, 5, 20):
        x_o, it_o, _, _ = oracle.cg_nb(A_o, b, maxit=k, tol=0.0)
        x_g, info = hs.cg_nb(A_g, dev(b), tol=0.0, maxit=k)
        assert info.iters == it_o == k
        assert rel(host(x_g), x_o) <= 1e-8, (k, rel(host(x_g), x_o))


@pytest.mark.parametrize("shape,kind", NB_CASES[:5])
def test_cg_nb_tolerance_mode(shape, kind):
    A_o, A_g, _k = make_ops(shape, kind)
    b = inputs.uniform_pm1(32, 1, A_o.N)
    tol = 1e-10
    _, it_o, st_o, _ = oracle.cg_nb(A_o, b, tol=tol, maxit=20000)
    _, it_c, _, _ = oracle.cg(A_o, b, tol=tol, maxit=20000)
    x_g, info = hs.cg_nb(A_g, dev(b), tol=tol, maxit=20000)
    assert st_o == oracle.OK and info.status == "OK"
    assert abs(it_o - it_c) <= 1, (it_o, it_c)
    # +-2 where the oracle's count is stable; var-k systems: the oracle's own
    # perturbation window (CG counts), one wider for CG-NB's different rounding
    lo, hi, counts, _, _ = oracle_window(A_o, b, "cg", it_c, tol)
    lo, hi = min(lo, it_o - 2) - 1, max(hi, it_o + 2) + 1
    assert lo <= info.iters <= hi, (info.iters, it_o, counts)
    assert A_o.relres(b, host(x_g)) <= tol * (1 + 1e-3)
    assert info.history[0] == pytest.approx(1.0) and info.history[info.iters] <= tol


def test_cg_nb_paper_order_final_step():
    A_o, A_g, _k = make_ops((70, 45), "lap")
    b = inputs.uniform_pm1(33, 1, A_o.N)
    x_o, it_o, _, _ = oracle.cg_nb(A_o, b, tol=1e-8, maxit=5000, paper_order=True)
    x_g, info = hs.cg_nb(A_g, dev(b), tol=1e-8, maxit=5000, paper_order=True)
    assert info.status == "OK" and abs(info.iters - it_o) <= 2
    # the returned iterate is one CG step beyond the converged one
    x_c, _, _, _ = oracle.cg(A_o, b, maxit=info.iters + 1, tol=0.0)
    assert rel(host(x_g), x_c) <= 1e-8
    assert A_o.relres(b, host(x_g)) < info.history[info.iters]


def test_cg_nb_edge_cases():
    A_o, A_g, _ = make_ops((20, 9, 7), "lap")
    b = torch.zeros(A_o.N, dtype=torch.float64, device="cuda")
    x, info = hs.cg_nb(A_g, b, torch.ones_like(b), tol=1e-8)
    assert info.status == "OK" and info.iters == 0 and torch.count_nonzero(x).item() == 0
    bb = dev(inputs.uniform_pm1(34, 1, A_o.N))
    x, info = hs.cg_nb(A_g, bb, tol=1e-14, maxit=4)
    assert info.status == "NOT_CONVERGED" and info.iters == 4
    bn = inputs.uniform_pm1(35, 1, A_o.N)
    bn[11] = np.nan
    x, info = hs.cg_nb(A_g, dev(bn), tol=1e-8, maxit=20)
    assert info.status == "ERR_NONFINITE"
    _, A_up, _ = make_ops((20, 9, 7), "up")
    with pytest.raises(hs.HsError):
        hs.cg_nb(A_up, bb, tol=1e-8)


def test_cg_nb_fp32():
    A_o, A_g, _ = make_ops((64, 33, 40), "lap")
    b = inputs.uniform_pm1(36, 1, A_o.N).astype(np.float32)
    x, info = hs.cg_nb(A_g, dev(b, torch.float32), tol=1e-5, maxit=5000)
    assert info.status == "OK"
    assert A_o.relres(b.astype(np.float64), host(x)) <= 2e-5


@pytest.mark.parametrize("shape,kind", [((70, 45), "up"), ((37, 19, 11), "up"), ((30, 22, 17), "vark")])
def test_bicgstab_b1_matches_oracle(shape, kind):
    A_o, A_g, _k = make_ops(shape, kind)
    b = inputs.uniform_pm1(37, 1, A_o.N)
    tol = 1e-9
    x_o, it_o, st_o, _, nr_o = oracle.bicgstab_b1(A_o, b, tol=tol, maxit=5000)
    x_g, info = hs.bicgstab(A_g, dev(b), tol=tol, maxit=5000, paper_order=True)
    assert st_o == oracle.OK and info.status == "OK"
    # +-2 where the oracle's B1 count is stable, else its measured range +-2
    lo, hi, counts, _, _ = oracle_window(A_o, b, "bicgstab_b1", it_o, tol)
    assert lo <= info.iters <= hi, (info.iters, counts, nr_o)
    assert A_o.relres(b, host(x_g)) <= tol * (1 + 1e-3)
    # B1 returns x_{l+1}: the classical iterate after as many iterations, to
    # 1e-8 or, where restarts make the count move, to the classical oracle's
    # own perturbed-run distance after that many iterations
    x_c, it_c, _, _, _ = oracle.bicgstab(A_o, b, tol=0.0, maxit=info.iters)
    assert it_c == info.iters
    xdev = oracle_xdev(A_o, b, "bicgstab", info.iters, x_c)
    err = rel(host(x_g), x_c)
    assert err <= iterate_bar(nr_o == 0, xdev), (err, xdev, nr_o)
