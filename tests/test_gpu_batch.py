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
        assert A_o.relres(b, xh) <= 1.5 * tol, (k, bsys)
        if bsys.solver == "cg":
            _, it_o, _, _ = oracle.cg(A_o, b, tol=tol, maxit=20000)
        else:
            _, it_o, _, _, _ = oracle.bicgstab(A_o, b, tol=tol, maxit=20000)
        # +-2 where the oracle's own count is stable, else its perturbation window
        lo, hi, counts = oracle_window(A_o, b, bsys.solver, it_o, tol)
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
    assert A_o.relres(bs[0].cpu().numpy(), xs[0].cpu().numpy()) <= 1.5e-8


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
        assert A_o.relres(b, x.cpu().numpy()) <= 1.5e-8


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
