"""Batched persistent solves: one cooperative kernel (replayed as a CUDA graph)
solves many independent systems of uneven sizes, each with its own
convergence test.  Every system is checked against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2305_05988_gb300 import inputs
from parity_util import oracle_window

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2305_05988_gb300 as hs  # noqa: E402


def build(systems, seed=0):
    ops_o, ops_g, bs, sol = [], [], [], []
    for bsys in systems:
        shape = bsys.shape
        if bsys.solver == "cg":
            ops_o.append(oracle.Operator(shape))
            ops_g.append(hs.Operator.laplacian(shape))
        else:
            beta = inputs.upwind_beta(shape, bsys.peclet)
            ops_o.append(oracle.Operator(shape, oracle.UPWIND, beta))
            ops_g.append(hs.Operator.upwind(shape, beta))
        b = inputs.uniform_pm1(seed, inputs.STREAM_BATCH_RHS + bsys.index, bsys.N)
        bs.append(b)
        sol.append(bsys.solver)
    return ops_o, ops_g, bs, sol


def small_batch(n=40, side_max=40, seed=5):
    return inputs.batch_systems(n, seed=seed, side_min=6, side_max=side_max)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_batch_matches_oracle_per_system():
    systems = small_batch()
    ops_o, ops_g, bs, sol = build(systems)
    batch = hs.Batch(ops_g, sol)
    tol = 1e-8
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        xs, infos = batch.solve([dev(b) for b in bs], tol=tol, maxit=20000)
    s.synchronize()
    for k, (A_o, b, x, info, bsys) in enumerate(zip(ops_o, bs, xs, infos, systems)):
        assert info.status == "OK", (k, bsys, info)
        xh = x.cpu().numpy()
        assert A_o.relres(b, xh) <= tol * (1 + 1e-3), (k, bsys)
        if bsys.solver == "cg":
            _, it_o, _, _ = oracle.cg(A_o, b, tol=tol, maxit=20000)
        else:
            _, it_o, _, _, _ = oracle.bicgstab(A_o, b, tol=tol, maxit=20000)
        # +-2 where the oracle's own count is stable, else its perturbation window
        lo, hi, counts, _, _ = oracle_window(A_o, b, bsys.solver, it_o, tol)
        assert lo <= info.iters <= hi, (k, bsys, info.iters, counts)


def test_batch_graph_replay_equals_direct_launch():
    systems = small_batch(24, 32, seed=9)
    _, ops_g, bs, sol = build(systems)
    batch = hs.Batch(ops_g, sol)
    bd = [dev(b) for b in bs]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        x1, i1 = batch.solve(bd, tol=1e-8, use_graph=True)
        g1 = batch.graph_used
        x2, i2 = batch.solve(bd, tol=1e-8, use_graph=True)
        g2 = batch.graph_used
        x3, i3 = batch.solve(bd, tol=1e-8, use_graph=False)
        g3 = batch.graph_used
    s.synchronize()
    assert g1 and g2 and not g3
    for a, b_, c in zip(x1, x2, x3):
        assert torch.equal(a, b_) and torch.equal(a, c)
    assert [i.iters for i in i1] == [i.iters for i in i2] == [i.iters for i in i3]


def test_batch_sizes_teams_by_work():
    shapes = [(96, 96, 96)] + [(8, 8)] * 30 + [(20, 20, 20)] * 5
    ops = [hs.Operator.laplacian(sh) for sh in shapes]
    batch = hs.Batch(ops, ["cg"] * len(ops))
    batch.workspace(torch.device("cuda"))
    teams = batch.teams
    assert teams[0] > 8 and all(t == 1 for t in teams[1:31])
    bs = [dev(inputs.uniform_pm1(1, 7, int(np.prod(sh)))) for sh in shapes]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        xs, infos = batch.solve(bs, tol=1e-8)
    s.synchronize()
    assert all(i.status == "OK" for i in infos)
    A_o = oracle.Operator(shapes[0])
    assert A_o.relres(bs[0].cpu().numpy(), xs[0].cpu().numpy()) <= 1e-8 * (1 + 1e-3)


def test_batch_poisoned_system_does_not_disturb_neighbours():
    systems = small_batch(16, 24, seed=11)
    ops_o, ops_g, bs, sol = build(systems)
    bad = 5
    bs[bad] = bs[bad].copy()
    bs[bad][3] = np.nan
    batch = hs.Batch(ops_g, sol)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        xs, infos = batch.solve([dev(b) for b in bs], tol=1e-8)
    s.synchronize()
    assert infos[bad].status == "ERR_NONFINITE"
    for k, (A_o, b, x, info) in enumerate(zip(ops_o, bs, xs, infos)):
        if k == bad:
            continue
        assert info.status == "OK"
        assert A_o.relres(b, x.cpu().numpy()) <= 1e-8 * (1 + 1e-3)


def test_batch_zero_rhs_and_maxit():
    shapes = [(12, 10), (9, 8, 7), (30,)]
    ops = [hs.Operator.laplacian(sh) for sh in shapes]
    batch = hs.Batch(ops, ["cg", "bicgstab", "cg"])
    bs = [torch.zeros(int(np.prod(sh)), dtype=torch.float64, device="cuda") for sh in shapes]
    bs[1] = dev(inputs.uniform_pm1(2, 7, 9 * 8 * 7))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        xs, infos = batch.solve(bs, xs=[torch.ones_like(b) for b in bs], tol=1e-12, maxit=3)
    s.synchronize()
    assert infos[0].status == "OK" and infos[0].iters == 0 and torch.count_nonzero(xs[0]).item() == 0
    assert infos[1].status == "NOT_CONVERGED" and infos[1].iters == 3


def build_mixed(systems, seed=0, vark_every=0):
    """Like build(), with every `vark_every`-th CG system on a variable-k
    diffusion operator (log k ~ N(0, 1))."""
    ops_o, ops_g, bs, ks = [], [], [], []
    for q, bsys in enumerate(systems):
        shape = bsys.shape
        if bsys.solver == "cg" and vark_every and q % vark_every == 0:
            k = np.exp(inputs.log_k(shape, 1.0, seed + q))
            ops_o.append(oracle.Operator(shape, oracle.DIFFUSION, k=k))
            kt = dev(k)
            ks.append(kt)
            ops_g.append(hs.Operator.diffusion(shape, kt))
        elif bsys.solver == "cg":
            ops_o.append(oracle.Operator(shape))
            ops_g.append(hs.Operator.laplacian(shape))
        else:
            beta = inputs.upwind_beta(shape, bsys.peclet)
            ops_o.append(oracle.Operator(shape, oracle.UPWIND, beta))
            ops_g.append(hs.Operator.upwind(shape, beta))
        bs.append(inputs.uniform_pm1(seed, inputs.STREAM_BATCH_RHS + bsys.index, bsys.N))
    return ops_o, ops_g, bs, ks


def test_batch_mixed_precision_certified_by_oracle():
    # FP64 refinement with FP32 inner solves reaches an FP64 residual of 1e-10
    # (below what FP32 alone can represent); the oracle's FP64 SpMV certifies
    # every system and its FP64 solution agrees to the conditioning bound
    systems = small_batch(24, 36, seed=13)
    ops_o, ops_g, bs, _ks = build_mixed(systems, vark_every=4)
    batch = hs.Batch(ops_g, ["mixed"] * len(ops_g))
    tol = 1e-10
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        xs, infos = batch.solve([dev(b) for b in bs], tol=tol, maxit=30, inner_tol=1e-4, inner_maxit=20000)
    s.synchronize()
    for k, (A_o, b, x, info, bsys) in enumerate(zip(ops_o, bs, xs, infos, systems)):
        assert info.status == "OK", (k, bsys, info)
        assert info.outer >= 2 and info.inner_iters > 0 and info.iters == info.outer, (k, info)
        xh = x.cpu().numpy()
        rr = A_o.relres(b, xh)
        assert rr <= tol * (1 + 1e-3), (k, bsys, rr)
        # the device's FP64 residual norm is the oracle's up to the rounding of b - A x
        assert abs(info.rel_res - rr) <= 0.05 * rr + 1e-13, (k, info.rel_res, rr)
        if bsys.solver == "cg":
            x_o, _, _, _ = oracle.cg(A_o, b, tol=1e-13, maxit=20000)
        else:
            x_o, _, _, _, _ = oracle.bicgstab(A_o, b, tol=1e-13, maxit=20000)
        # ||x - x*|| / ||x*|| <= cond(A) * ||r|| / ||b||; cond <= 4 (n+1)^2 / pi^2 for these grids
        n = max(bsys.shape)
        bound = 4.0 * (n + 1) ** 2 / np.pi ** 2 * 1e-10 * 10
        assert np.linalg.norm(xh - x_o) <= bound * np.linalg.norm(x_o), (k, bsys)


def test_batch_mixed_matches_standalone_mixed_counts():
    # one system alone in a batch runs the standalone refinement's arithmetic
    # up to the power-of-two residual scaling: same outer steps, inner counts
    # within a few iterations
    shape = (40, 36, 30)
    A = hs.Operator.laplacian(shape)
    b = dev(inputs.uniform_pm1(0, 77, int(np.prod(shape))))
    batch = hs.Batch([A], ["mixed"])
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        xb, ib = batch.solve([b], tol=1e-10, maxit=20, inner_tol=1e-4)
        xs, info = hs.solve_mixed(A, b, tol=1e-10, maxit=20, inner_tol=1e-4)
    s.synchronize()
    assert ib[0].status == "OK" and info.status == "OK"
    assert ib[0].outer == info.outer
    assert abs(ib[0].inner_iters - info.inner_iters) <= 3 * info.outer, (ib[0], info)
    assert torch.linalg.norm(xb[0] - xs).item() <= 1e-8 * torch.linalg.norm(xs).item()


def test_batch_mixed_adaptive_inner_tolerance():
    # the mixed batch applies the same rule as the standalone refinement: a
    # step close to tol runs its inner solve only to 0.5 tol / rel; fewer inner
    # iterations in total, every system still certified by the oracle
    systems = small_batch(12, 36, seed=17)
    ops_o, ops_g, bs, _ks = build_mixed(systems, vark_every=3)
    batch = hs.Batch(ops_g, ["mixed"] * len(ops_g))
    tol = 1e-10
    s = torch.cuda.Stream()
    runs = {}
    for fixed in (1, 0):
        with torch.cuda.stream(s):
            xs, infos = batch.solve([dev(b) for b in bs], tol=tol, maxit=30, inner_tol=1e-4, inner_maxit=20000,
                                    inner_fixed_tol=fixed)
        s.synchronize()
        for A_o, b, x, info in zip(ops_o, bs, xs, infos):
            assert info.status == "OK", info
            assert A_o.relres(b, x.cpu().numpy()) <= tol * (1 + 1e-3)
        runs[fixed] = infos
    assert sum(i.inner_iters for i in runs[0]) <= sum(i.inner_iters for i in runs[1])


def test_batch_mixed_poisoned_and_all_or_none():
    systems = small_batch(12, 20, seed=17)
    ops_o, ops_g, bs, _ = build_mixed(systems)
    bad = 3
    bs[bad] = bs[bad].copy()
    bs[bad][5] = np.inf
    batch = hs.Batch(ops_g, ["mixed"] * len(ops_g))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        xs, infos = batch.solve([dev(b) for b in bs], tol=1e-10, maxit=30, inner_tol=1e-4)
    s.synchronize()
    assert infos[bad].status == "ERR_NONFINITE"
    for k, (A_o, b, x, info) in enumerate(zip(ops_o, bs, xs, infos)):
        if k != bad:
            assert info.status == "OK" and A_o.relres(b, x.cpu().numpy()) <= 1e-10 * (1 + 1e-3)
    with pytest.raises(hs.HsError):
        hs.Batch(ops_g[:2], ["mixed", "cg"])


def test_batch_solve_function():
    # the one-call form: builds the batch and solves; each system against the oracle
    shapes = [(20, 18), (12, 10, 9), (30, 7), (9, 9, 9)]
    ops_o, ops_g, bs, sol = [], [], [], []
    for q, shape in enumerate(shapes):
        if q % 2 == 0:
            ops_o.append(oracle.Operator(shape))
            ops_g.append(hs.Operator.laplacian(shape))
            sol.append("cg")
        else:
            beta = inputs.upwind_beta(shape, 0.5)
            ops_o.append(oracle.Operator(shape, oracle.UPWIND, beta))
            ops_g.append(hs.Operator.upwind(shape, beta))
            sol.append("bicgstab")
        bs.append(inputs.uniform_pm1(70 + q, 1, int(np.prod(shape))))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        xs, infos = hs.batch_solve(ops_g, sol, [dev(b) for b in bs], tol=1e-10, maxit=5000)
    s.synchronize()
    for A_o, b, x, info in zip(ops_o, bs, xs, infos):
        assert info.status == "OK"
        assert A_o.relres(b, x.cpu().numpy()) <= 1e-10 * (1 + 1e-3)
