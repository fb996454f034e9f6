"""Pins of the FP64 CPU oracle against facts that do not come from the oracle.

Each test names what fixes the expected value: an independent Kronecker-sum
assembly, a closed-form eigenpair, a dense LU / triangular solve (numpy,
scipy), an exact property of the method in exact arithmetic, or a finite
difference through dense solves.  A plausible slip in the oracle (a dropped
term, a wrong sign or index, a transposed operand, a wrong stopping rule)
makes at least one of them fail.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from dense_ref import (grid_coords, kron_sum, laplacian_dense, tensor_vec, toeplitz_eig_1d, tridiag,
                       upwind_dense)
from paper_2305_05988_gb300 import inputs

TINY_SHAPES = [(1,), (7,), (1, 1), (2, 3), (5, 4), (3, 4, 5), (2, 1, 3)]


def unit_columns(A):
    """Dense matrix of an oracle operator recovered through its SpMV alone."""
    M = np.zeros((A.N, A.N))
    for j in range(A.N):
        e = np.zeros(A.N)
        e[j] = 1.0
        M[:, j] = A.spmv(e)
    return M


# --------------------------------------------------------------------------
# Operators / SpMV
# --------------------------------------------------------------------------

@pytest.mark.parametrize("shape", TINY_SHAPES)
def test_laplacian_matches_kronecker_sum(shape):
    A = oracle.Operator(shape)
    M = unit_columns(A)
    ref = laplacian_dense(shape)
    assert np.allclose(M, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    assert np.array_equal(A.dense(), M)


@pytest.mark.parametrize("shape", [(6,), (5, 4), (3, 4, 5)])
def test_upwind_matches_kronecker_sum(shape):
    beta = inputs.upwind_beta(shape, 0.5)
    A = oracle.Operator(shape, oracle.UPWIND, beta)
    M = unit_columns(A)
    ref = upwind_dense(shape, beta)
    assert np.allclose(M, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    # upwind: the lower neighbour carries the convection term, so A is not symmetric
    assert not np.allclose(M, M.T)


@pytest.mark.parametrize("shape", [(9, 7), (6, 5, 4), (128, 128)])
@pytest.mark.parametrize("modes", [(1, 1, 1), (2, 3, 1), (3, 1, 2)])
def test_laplacian_closed_form_eigenpairs(shape, modes):
    # v = prod sin(p_d pi x_d), lambda = sum (4/h_d^2) sin^2(p_d pi h_d / 2)
    xs = grid_coords(shape)
    v = np.ones(int(np.prod(shape)))
    lam = 0.0
    for d, n in enumerate(shape):
        p = modes[d]
        h = 1.0 / (n + 1)
        v *= np.sin(p * math.pi * xs[d])
        lam += 4.0 / h**2 * math.sin(p * math.pi * h / 2) ** 2
    A = oracle.Operator(shape)
    Av = A.spmv(v)
    assert np.linalg.norm(Av - lam * v) <= 1e-13 * lam * np.linalg.norm(v) * 10


@pytest.mark.parametrize("shape", [(8,), (6, 5), (5, 4, 6)])
def test_upwind_toeplitz_eigenpairs(shape):
    beta = inputs.upwind_beta(shape, 0.5)
    A = oracle.Operator(shape, oracle.UPWIND, beta)
    vs, lam = [], 0.0
    for d, n in enumerate(shape):
        h = 1.0 / (n + 1)
        lo, dg, up = -1.0 / h**2 - beta[d] / h, 2.0 / h**2 + beta[d] / h, -1.0 / h**2
        l1, v1 = toeplitz_eig_1d(n, lo, dg, up, m=1 + d)
        vs.append(v1)
        lam += l1
    v = tensor_vec(vs)
    Av = A.spmv(v)
    assert np.linalg.norm(Av - lam * v) <= 1e-12 * abs(lam) * np.linalg.norm(v)


def test_diffusion_constant_k_is_scaled_laplacian():
    shape = (4, 3, 5)
    for c in (1.0, 2.5):
        A = oracle.Operator(shape, oracle.DIFFUSION, k=np.full(60, c))
        ref = c * laplacian_dense(shape)
        assert np.allclose(unit_columns(A), ref, rtol=1e-14, atol=1e-12 * np.abs(ref).max())


def test_diffusion_alternating_k_closed_form_1d():
    # k alternating 1, 3: every interior face has harmonic mean 2*1*3/4 = 1.5;
    # the boundary faces take the cell's own k (first cell 1, last cell k[-1]).
    n = 6
    k = np.array([1.0, 3.0] * 3)
    h = 1.0 / (n + 1)
    A = oracle.Operator((n,), oracle.DIFFUSION, k=k)
    M = unit_columns(A)
    ref = tridiag(n, -1.5, 3.0, -1.5)
    ref[0, 0] = 1.5 + k[0]
    ref[-1, -1] = 1.5 + k[-1]
    assert np.allclose(M, ref / h**2, rtol=1e-14)


def test_diffusion_quadratic_form_and_symmetry():
    # x^T A x = sum_interior faces kappa (x_i - x_j)^2 / h^2 + sum_boundary faces k_i x_i^2 / h^2
    shape = (3, 4, 2)
    N = 24
    k = np.exp(inputs.normal(3, inputs.STREAM_K, N))
    A = oracle.Operator(shape, oracle.DIFFUSION, k=k)
    M = unit_columns(A)
    assert np.allclose(M, M.T, rtol=1e-14, atol=0)
    x = inputs.uniform_pm1(4, 1, N)
    q = 0.0
    kk = k.reshape(shape[::-1])  # [z, y, x]
    xx = x.reshape(shape[::-1])
    h = [1.0 / (n + 1) for n in shape]
    for ax, d in ((2, 0), (1, 1), (0, 2)):
        a, b = np.moveaxis(kk, ax, 0), np.moveaxis(xx, ax, 0)
        kap = 2 * a[:-1] * a[1:] / (a[:-1] + a[1:])
        q += np.sum(kap * (b[:-1] - b[1:]) ** 2) / h[d] ** 2
        q += (np.sum(a[0] * b[0] ** 2) + np.sum(a[-1] * b[-1] ** 2)) / h[d] ** 2
    assert abs(x @ M @ x - q) <= 1e-12 * abs(q)
    assert np.all(np.linalg.eigvalsh(M) > 0)


def test_dot_is_nearly_correctly_rounded():
    # math.fsum is the correctly rounded sum of the rounded products; the
    # oracle's inner product must sit within 2 ulps of it, even where plain
    # left-to-right summation cancels catastrophically.
    a = np.array([1e16, 1.0, -1e16, 3.0])
    b = np.ones(4)
    assert oracle.dot(a, b) == 4.0
    rng = np.random.default_rng(0)
    for n in (1, 17, 1000, 100000):
        x = rng.standard_normal(n) * np.exp(rng.uniform(-20, 20, n))
        y = rng.standard_normal(n)
        ref = math.fsum((x * y).tolist())
        assert abs(oracle.dot(x, y) - ref) <= 2 * np.spacing(abs(ref)) + 1e-300


# --------------------------------------------------------------------------
# Jacobi
# --------------------------------------------------------------------------

@pytest.mark.parametrize("shape,sweeps", [((128, 128), 500), ((24, 24, 24), 200), ((9, 13), 50)])
def test_jacobi_closed_form_lowest_mode(shape, sweeps):
    # b = lambda v for the lowest mode; D constant -> x_k = (1 - mu^k) v, mu = 1 - lambda/D
    xs = grid_coords(shape)
    v = np.ones(int(np.prod(shape)))
    lam, D = 0.0, 0.0
    for d, n in enumerate(shape):
        h = 1.0 / (n + 1)
        v *= np.sin(math.pi * xs[d])
        lam += 4.0 / h**2 * math.sin(math.pi * h / 2) ** 2
        D += 2.0 / h**2
    mu = 1.0 - lam / D
    if len(set(shape)) == 1:
        assert abs(mu - math.cos(math.pi / (shape[0] + 1))) < 1e-13
    A = oracle.Operator(shape)
    x, it, st, _ = oracle.jacobi(A, lam * v, maxit=sweeps)
    assert it == sweeps and st == oracle.OK
    ref = (1.0 - mu**sweeps) * v
    # rounding bound: each sweep rounds every entry (2d + 2) times at unit
    # roundoff u, and the lowest mode barely decays, so errors add over k sweeps
    bound = sweeps * (2 * len(shape) + 2) * 2.0**-53
    assert np.linalg.norm(x - ref) <= bound * np.linalg.norm(ref)


@pytest.mark.parametrize("shape,kind", [((5, 4), "lap"), ((3, 4, 5), "lap"), ((4, 5), "up"), ((3, 3, 4), "up")])
def test_jacobi_dense_recurrence(shape, kind):
    N = int(np.prod(shape))
    if kind == "lap":
        M = laplacian_dense(shape)
        A = oracle.Operator(shape)
    else:
        beta = inputs.upwind_beta(shape, 0.5)
        M = upwind_dense(shape, beta)
        A = oracle.Operator(shape, oracle.UPWIND, beta)
    b = inputs.uniform_pm1(7, 1, N)
    Dg = np.diag(M)
    R = M - np.diag(Dg)
    x = np.zeros(N)
    for _ in range(13):
        x = (b - R @ x) / Dg
    xo, it, _, _ = oracle.jacobi(A, b, maxit=13)
    assert np.linalg.norm(xo - x) <= 1e-14 * np.linalg.norm(x)


def test_jacobi_tolerance_stops_at_first_iterate_below_tol():
    shape = (12, 10)
    A = oracle.Operator(shape)
    b = inputs.rhs_uniform(shape, 1)
    x, it, st, hist = oracle.jacobi(A, b, maxit=5000, tol=1e-3, history=True)
    assert st == oracle.OK
    assert hist[it] <= 1e-3 < hist[it - 1]
    assert abs(A.relres(b, x) - hist[it]) < 1e-15
    # each entry of the history is the true relative residual of that iterate
    x5, _, _, _ = oracle.jacobi(A, b, maxit=5)
    assert abs(A.relres(b, x5) - hist[5]) < 1e-15


# --------------------------------------------------------------------------
# Gauss-Seidel
# --------------------------------------------------------------------------

@pytest.mark.parametrize("shape,kind", [((5, 4), "lap"), ((3, 4, 5), "lap"), ((4, 5), "up"), ((3, 3, 4), "up"),
                                        ((7,), "lap"), ((1, 1), "lap")])
def test_gs_dense_triangular(shape, kind):
    N = int(np.prod(shape))
    if kind == "lap":
        M = laplacian_dense(shape)
        A = oracle.Operator(shape)
    else:
        beta = inputs.upwind_beta(shape, 0.5)
        M = upwind_dense(shape, beta)
        A = oracle.Operator(shape, oracle.UPWIND, beta)
    b = inputs.uniform_pm1(9, 1, N)
    L = np.tril(M)            # D + L
    U = np.triu(M)            # D + U
    x = inputs.uniform_pm1(10, 1, N)
    fwd = sla.solve_triangular(L, b - np.triu(M, 1) @ x, lower=True)
    got = oracle.gs_sweep(A, b, x)
    assert np.linalg.norm(got - fwd) <= 1e-14 * max(1.0, np.linalg.norm(fwd))
    bwd = sla.solve_triangular(U, b - np.tril(M, -1) @ x, lower=False)
    got = oracle.gs_sweep(A, b, x, backward=True)
    assert np.linalg.norm(got - bwd) <= 1e-14 * max(1.0, np.linalg.norm(bwd))
    # symmetric = forward then backward
    sym = sla.solve_triangular(U, b - np.tril(M, -1) @ fwd, lower=False)
    xs, it, _, _ = oracle.gauss_seidel(A, b, x, maxit=1, mode=oracle.GS_SYMMETRIC)
    assert np.linalg.norm(xs - sym) <= 1e-14 * max(1.0, np.linalg.norm(sym))
    # several forward sweeps
    y = x.copy()
    for _ in range(6):
        y = sla.solve_triangular(L, b - np.triu(M, 1) @ y, lower=True)
    xf, _, _, _ = oracle.gauss_seidel(A, b, x, maxit=6, mode=oracle.GS_FORWARD)
    assert np.linalg.norm(xf - y) <= 1e-13 * max(1.0, np.linalg.norm(y))


def test_gs_asymptotic_rate_is_jacobi_rate_squared():
    # Young: for the consistently ordered model matrix rho(GS) = rho(J)^2 = cos^2(pi h)
    shape = (15, 15)
    M = laplacian_dense(shape)
    b = inputs.rhs_uniform(shape, 2)
    xs = np.linalg.solve(M, b)
    A = oracle.Operator(shape)
    x1, _, _, _ = oracle.gauss_seidel(A, b, maxit=700)
    x2, _, _, _ = oracle.gauss_seidel(A, b, x1, maxit=1)
    ratio = np.linalg.norm(x2 - xs) / np.linalg.norm(x1 - xs)
    assert abs(ratio - math.cos(math.pi / 16) ** 2) < 2e-3


# --------------------------------------------------------------------------
# CG
# --------------------------------------------------------------------------

def test_cg_manufactured_eigenvector_one_iteration():
    shape = (128, 128)
    f = inputs.rhs_manufactured_2d(shape)
    A = oracle.Operator(shape)
    x, it, st, hist = oracle.cg(A, f, tol=1e-10)
    h = 1.0 / 129
    lam = 2 * 4.0 / h**2 * math.sin(math.pi * h / 2) ** 2
    xs, ys = grid_coords(shape)
    exact = (2 * math.pi**2 / lam) * np.sin(math.pi * xs) * np.sin(math.pi * ys)
    assert st == oracle.OK and it == 1
    assert np.linalg.norm(x - exact) <= 1e-13 * np.linalg.norm(exact)


@pytest.mark.parametrize("shape", [(5, 4), (3, 4, 5), (9,), (6, 6)])
def test_cg_dense_lu(shape):
    M = laplacian_dense(shape)
    N = M.shape[0]
    b = inputs.uniform_pm1(11, 1, N)
    ref = sla.lu_solve(sla.lu_factor(M), b)
    x, it, st, hist = oracle.cg(oracle.Operator(shape), b, maxit=200, tol=1e-13)
    assert st == oracle.OK
    assert np.linalg.norm(x - ref) <= 1e-12 * np.linalg.norm(ref)
    assert np.all(np.diff(hist) != 0)


@pytest.mark.parametrize("shape", [(4, 4), (3, 3, 3), (6, 4)])
def test_cg_finite_termination(shape):
    M = laplacian_dense(shape)
    ev = np.linalg.eigvalsh(M)
    distinct = len(np.unique(np.round(ev / ev.max(), 10)))
    b = inputs.uniform_pm1(12, 1, M.shape[0])
    x, it, st, hist = oracle.cg(oracle.Operator(shape), b, maxit=100, tol=1e-11)
    assert st == oracle.OK and it <= distinct


def test_cg_residual_orthogonality_and_conjugacy():
    shape = (7, 6)
    M = laplacian_dense(shape)
    N = M.shape[0]
    b = inputs.uniform_pm1(13, 1, N)
    A = oracle.Operator(shape)
    xs = [np.zeros(N)]
    for m in range(1, 7):
        x, it, _, _ = oracle.cg(A, b, maxit=m, tol=0.0)
        assert it == m
        xs.append(x)
    rs = [b - M @ x for x in xs]
    ps = [xs[i + 1] - xs[i] for i in range(len(xs) - 1)]
    for i in range(len(rs)):
        for j in range(i):
            c = abs(rs[i] @ rs[j]) / (np.linalg.norm(rs[i]) * np.linalg.norm(rs[j]))
            assert c < 1e-10
    for i in range(len(ps)):
        for j in range(i):
            c = abs(ps[i] @ M @ ps[j]) / math.sqrt((ps[i] @ M @ ps[i]) * (ps[j] @ M @ ps[j]))
            assert c < 1e-10


def test_cg_zero_rhs_and_history():
    A = oracle.Operator((6, 5))
    x, it, st, hist = oracle.cg(A, np.zeros(30), x0=np.ones(30))
    assert it == 0 and st == oracle.OK and np.all(x == 0)
    b = inputs.rhs_uniform((6, 5), 3)
    x, it, st, hist = oracle.cg(A, b, maxit=3, tol=1e-14)
    assert st == oracle.NOT_CONVERGED and it == 3 and hist[0] == 1.0
    assert abs(hist[3] - A.relres(b, x)) < 1e-12


# --------------------------------------------------------------------------
# BiCGStab
# --------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(6, 5), (3, 4, 5), (10,)])
def test_bicgstab_dense_lu_upwind(shape):
    beta = inputs.upwind_beta(shape, 0.5)
    M = upwind_dense(shape, beta)
    b = inputs.uniform_pm1(14, 1, M.shape[0])
    ref = sla.lu_solve(sla.lu_factor(M), b)
    for eps in (1e-5, 0.0):
        x, it, st, hist, nr = oracle.bicgstab(oracle.Operator(shape, oracle.UPWIND, beta), b,
                                              maxit=500, tol=1e-13, restart_eps=eps)
        assert st == oracle.OK
        assert np.linalg.norm(x - ref) <= 1e-11 * np.linalg.norm(ref)


def test_bicgstab_eigenvector_rhs_one_iteration():
    shape = (8, 7)
    beta = inputs.upwind_beta(shape, 0.7)
    vs, lam = [], 0.0
    for d, n in enumerate(shape):
        h = 1.0 / (n + 1)
        l1, v1 = toeplitz_eig_1d(n, -1.0 / h**2 - beta[d] / h, 2.0 / h**2 + beta[d] / h, -1.0 / h**2, 2)
        vs.append(v1)
        lam += l1
    v = tensor_vec(vs)
    x, it, st, _, _ = oracle.bicgstab(oracle.Operator(shape, oracle.UPWIND, beta), lam * v, tol=1e-12)
    assert st == oracle.OK and it == 1
    assert np.linalg.norm(x - v) <= 1e-13 * np.linalg.norm(v)


def test_bicgstab_on_spd_reaches_cg_solution():
    shape = (20, 17)
    A = oracle.Operator(shape)
    b = inputs.rhs_uniform(shape, 5)
    xc, _, _, _ = oracle.cg(A, b, tol=1e-12, maxit=2000)
    xb, it, st, hist, _ = oracle.bicgstab(A, b, tol=1e-12, maxit=2000)
    assert st == oracle.OK
    assert np.linalg.norm(xb - xc) <= 1e-9 * np.linalg.norm(xc)
    assert hist[it] <= 1e-12
    assert A.relres(b, xb) <= 2e-12


def test_bicgstab_restart_fires_and_both_converge():
    # A tiny restart threshold never fires; a large one fires every iteration
    # and degrades to restarted minimal-residual steps; both must converge.
    shape = (16, 12)
    beta = inputs.upwind_beta(shape, 0.5)
    A = oracle.Operator(shape, oracle.UPWIND, beta)
    b = inputs.rhs_uniform(shape, 6)
    ref = np.linalg.solve(upwind_dense(shape, beta), b)
    x0, it0, st0, _, nr0 = oracle.bicgstab(A, b, tol=1e-11, maxit=3000, restart_eps=0.0)
    x1, it1, st1, _, nr1 = oracle.bicgstab(A, b, tol=1e-11, maxit=3000, restart_eps=1e3)
    assert nr0 == 0 and nr1 > 0
    assert st0 == oracle.OK and st1 == oracle.OK
    for x in (x0, x1):
        assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)


def test_bicgstab_trace_is_the_shadow_residual_product():
    # trace[k] = r_k . r' with r' = r_0 / ||r_0|| before any restart; computed
    # here from the iterates with a dense matrix and numpy, not the oracle's
    # recursion.  With restarts on every iteration (eps' = 1e3) the shadow
    # residual of iteration k + 1 is r_k / ||r_k||.
    shape = (9, 7, 5)
    beta = inputs.upwind_beta(shape, 0.5)
    A = oracle.Operator(shape, oracle.UPWIND, beta)
    M = upwind_dense(shape, beta)
    b = inputs.rhs_uniform(shape, 8)
    r0 = b.copy()
    rs = r0 / np.linalg.norm(r0)
    _, it, _, _, tr, at = oracle.bicgstab_trace(A, b, tol=1e-12, maxit=400, restart_eps=0.0)
    assert at == [] and np.isclose(tr[0], np.linalg.norm(r0), rtol=1e-14)
    for k in (1, 2, 3, 5):
        xk = oracle.bicgstab(A, b, tol=0.0, maxit=k, restart_eps=0.0)[0]
        assert np.isclose(tr[k], (b - M @ xk) @ rs, rtol=1e-9, atol=1e-12 * np.linalg.norm(r0))
    _, it, _, _, tr, at = oracle.bicgstab_trace(A, b, tol=1e-12, maxit=400, restart_eps=1e3)
    assert at == list(range(1, it))
    for k in (1, 2, 4):
        xk = oracle.bicgstab(A, b, tol=0.0, maxit=k, restart_eps=1e3)[0]
        xk1 = oracle.bicgstab(A, b, tol=0.0, maxit=k + 1, restart_eps=1e3)[0]
        rk = b - M @ xk
        assert np.isclose(tr[k + 1], (b - M @ xk1) @ (rk / np.linalg.norm(rk)), rtol=1e-7,
                          atol=1e-11 * np.linalg.norm(r0))


def test_bicgstab_restart_iterations_follow_the_threshold():
    shape = (70, 45)
    A = oracle.Operator(shape, oracle.UPWIND, inputs.upwind_beta(shape, 0.5))
    b = inputs.uniform_pm1(12, 1, A.N)
    _, it, st, _, tr, at = oracle.bicgstab_trace(A, b, tol=1e-10, maxit=5000, restart_eps=1e-5)
    _, it2, _, _, nr = oracle.bicgstab(A, b, tol=1e-10, maxit=5000, restart_eps=1e-5)
    assert st == oracle.OK and it == it2 and len(at) == nr > 0
    below = [k for k in range(1, it) if math.sqrt(abs(tr[k])) < 1e-5]
    assert below == at


def test_all_cores_build_is_bitwise_the_sequential_one():
    if not oracle.have_all_cores():
        pytest.skip("gcc without OpenMP")
    shape = (33, 21, 17)
    N = int(np.prod(shape))
    k = np.exp(inputs.normal(3, inputs.STREAM_K, N, 1.0))
    ops = [oracle.Operator(shape), oracle.Operator(shape, oracle.UPWIND, inputs.upwind_beta(shape, 0.5)),
           oracle.Operator(shape, oracle.DIFFUSION, k=k)]
    b = inputs.uniform_pm1(4, 1, N)

    def run():
        out = []
        for A in ops:
            out.append(A.spmv(b))
            out.append(oracle.jacobi(A, b, maxit=7)[0])
            out.append(oracle.bicgstab(A, b, tol=1e-10, maxit=500)[0])
            out.append(oracle.cg_nb(ops[0], b, tol=1e-10, maxit=500)[0])
        out.append(oracle.cg(ops[2], b, tol=1e-10, maxit=2000)[0])
        out.append(oracle.grad_logk(ops[2], out[0], out[1]))
        return out

    seq = run()
    with oracle.all_cores(4) as n:
        assert n == 4
        par = run()
    for a, c in zip(seq, par):
        assert np.array_equal(a, c)


# --------------------------------------------------------------------------
# HPCG 7- and 27-point systems (section 4.1)
# --------------------------------------------------------------------------

def hpcg27_dense(shape):
    """28 I - T_z (x) T_y (x) T_x with T = tridiag(1, 1, 1): -1 on the 26
    neighbours of the 3x3x3 box inside the grid, 27 on the diagonal."""
    Ts = [tridiag(n, 1.0, 1.0, 1.0) for n in shape]
    K = Ts[-1]
    for T in reversed(Ts[:-1]):
        K = np.kron(K, T)
    return 28.0 * np.eye(K.shape[0]) - K


def hpcg7_dense(shape):
    """27 I - (B_x (+) B_y (+) B_z) with B = tridiag(1, 0, 1)."""
    return 27.0 * np.eye(int(np.prod(shape))) - kron_sum([tridiag(n, 1.0, 0.0, 1.0) for n in shape])


@pytest.mark.parametrize("shape", [(3, 4, 5), (2, 2, 2), (5, 1, 3), (4, 3)])
def test_hpcg_dense_assembly(shape):
    for kind, ref in ((oracle.HPCG27, hpcg27_dense), (oracle.HPCG7, hpcg7_dense)):
        if kind == oracle.HPCG27 and len(shape) < 3:
            continue
        M = oracle.Operator(shape, kind).dense()
        assert np.array_equal(M, ref(shape))
        x = inputs.uniform_pm1(41, 1, M.shape[0])
        assert np.allclose(oracle.Operator(shape, kind).spmv(x), M @ x, rtol=0, atol=1e-13)


def test_hpcg27_closed_form_eigenpairs():
    # T = tridiag(1,1,1) has eigenpairs 1 + 2 cos(m pi/(n+1)), sin(i m pi/(n+1))
    shape = (9, 7, 6)
    A = oracle.Operator(shape, oracle.HPCG27)
    for ms in ((1, 1, 1), (2, 5, 3), (9, 7, 6)):
        vs, prod = [], 1.0
        for n, m in zip(shape, ms):
            th = m * math.pi / (n + 1)
            vs.append(np.sin(th * np.arange(1, n + 1)))
            prod *= 1.0 + 2.0 * math.cos(th)
        v = tensor_vec(vs)
        lam = 28.0 - prod
        assert np.linalg.norm(A.spmv(v) - lam * v) <= 1e-13 * np.linalg.norm(v) * 28


def test_hpcg_exact_solution_ones():
    # b = A 1 makes x = 1 the exact solution (section 4.1); every interior
    # row of the 27-point system sums to 1, of the 7-point one to 21
    shape = (12, 10, 9)
    for kind, interior in ((oracle.HPCG27, 1.0), (oracle.HPCG7, 21.0)):
        A = oracle.Operator(shape, kind)
        b = A.spmv(np.ones(A.N))
        assert b.reshape(9, 10, 12)[4, 5, 6] == interior
        x, it, st, _ = oracle.cg(A, b, tol=1e-13, maxit=500)
        assert st == oracle.OK and np.max(np.abs(x - 1.0)) <= 1e-12
        xb, _, stb, _, _ = oracle.bicgstab(A, b, tol=1e-13, maxit=500)
        assert stb == oracle.OK and np.max(np.abs(xb - 1.0)) <= 1e-12
        xj, _, _, _ = oracle.jacobi(A, b, maxit=2000, tol=1e-14)
        assert np.max(np.abs(xj - 1.0)) <= 1e-12


@pytest.mark.parametrize("ms,sweeps", [((1, 1, 1), 60), ((3, 2, 4), 25)])
def test_hpcg27_jacobi_closed_form(ms, sweeps):
    # D = 27 I: for b = lambda v (v an eigenvector of A) and x0 = 0 the Jacobi
    # error contracts by mu = 1 - lambda/27 per sweep, x_k = (1 - mu^k) v
    shape = (9, 7, 6)
    A = oracle.Operator(shape, oracle.HPCG27)
    vs, prod = [], 1.0
    for n, m in zip(shape, ms):
        th = m * math.pi / (n + 1)
        vs.append(np.sin(th * np.arange(1, n + 1)))
        prod *= 1.0 + 2.0 * math.cos(th)
    v = tensor_vec(vs)
    lam = 28.0 - prod
    mu = 1.0 - lam / 27.0
    x, it, _, _ = oracle.jacobi(A, lam * v, maxit=sweeps)
    assert it == sweeps
    ref = (1.0 - mu ** sweeps) * v
    assert np.linalg.norm(x - ref) <= 1e-12 * np.linalg.norm(ref)


def test_hpcg27_krylov_one_step_on_an_eigenvector():
    # b = v with A v = lambda v: the first Krylov space holds x* = v / lambda
    shape = (9, 7, 6)
    A = oracle.Operator(shape, oracle.HPCG27)
    vs, prod = [], 1.0
    for n, m in zip(shape, (2, 3, 1)):
        th = m * math.pi / (n + 1)
        vs.append(np.sin(th * np.arange(1, n + 1)))
        prod *= 1.0 + 2.0 * math.cos(th)
    v = tensor_vec(vs)
    lam = 28.0 - prod
    x, it, st, _ = oracle.cg(A, v, tol=1e-12, maxit=10)
    assert st == oracle.OK and it == 1
    assert np.linalg.norm(x - v / lam) <= 1e-13 * np.linalg.norm(v / lam)
    xb, itb, stb, _, _ = oracle.bicgstab(A, v, tol=1e-12, maxit=10)
    assert stb == oracle.OK and itb == 1
    assert np.linalg.norm(xb - v / lam) <= 1e-13 * np.linalg.norm(v / lam)


@pytest.mark.parametrize("shape", [(4, 3, 5), (3, 3, 3)])
def test_hpcg27_gauss_seidel_dense_triangular(shape):
    # forward: (D + L) x' = b - U x; backward: (D + U) x' = b - L x
    M = hpcg27_dense(shape)
    N = M.shape[0]
    Lw, Up = np.tril(M), np.triu(M, 1)
    b = inputs.uniform_pm1(44, 1, N)
    x0 = inputs.uniform_pm1(45, 1, N)
    A = oracle.Operator(shape, oracle.HPCG27)
    x1 = oracle.gs_sweep(A, b, x0)
    ref = sla.solve_triangular(Lw, b - Up @ x0, lower=True)
    assert np.linalg.norm(x1 - ref) <= 1e-14 * np.linalg.norm(ref)
    xb, _, _, _ = oracle.gauss_seidel(A, b, x0, maxit=1, mode=oracle.GS_BACKWARD)
    refb = sla.solve_triangular(np.triu(M), b - np.tril(M, -1) @ x0, lower=False)
    assert np.linalg.norm(xb - refb) <= 1e-14 * np.linalg.norm(refb)


# --------------------------------------------------------------------------
# CG-NB (Algorithm 1) and BiCGStab-B1 (Algorithm 2's statement order)
# --------------------------------------------------------------------------

# 1-D grids are left out: there CG terminates (residual at rounding level)
# and Algorithm 1's x update, which divides by alpha_n,j, turns the rounding
# noise of p_j - r_j into an O(1e-4) error (a property of the printed update).
@pytest.mark.parametrize("shape", [(5, 4), (3, 4, 5), (12, 11), (6, 6)])
def test_cg_nb_dense_lu(shape):
    M = laplacian_dense(shape)
    b = inputs.uniform_pm1(21, 1, M.shape[0])
    ref = sla.lu_solve(sla.lu_factor(M), b)
    x, it, st, hist = oracle.cg_nb(oracle.Operator(shape), b, maxit=200, tol=1e-13)
    assert st == oracle.OK
    assert np.linalg.norm(x - ref) <= 1e-12 * np.linalg.norm(ref)


def test_cg_nb_equals_classical_cg_iterates():
    # arithmetically equivalent to CG (section 3.2): the same iterate after k
    # iterations up to rounding.  A wrong sign in the x update (the printed
    # minus) would move x away from the CG iterate by 2 alpha p per step.
    shape = (23, 17)
    A = oracle.Operator(shape)
    b = inputs.rhs_uniform(shape, 7)
    for k in (1, 2, 5, 20, 60):
        xc, itc, _, _ = oracle.cg(A, b, maxit=k, tol=0.0)
        xn, itn, _, _ = oracle.cg_nb(A, b, maxit=k, tol=0.0)
        assert itc == itn == k
        assert np.linalg.norm(xn - xc) <= 1e-10 * np.linalg.norm(xc), k


def test_cg_nb_equals_classical_cg_on_the_27_point_system():
    shape = (9, 8, 7)
    A = oracle.Operator(shape, oracle.HPCG27)
    b = A.spmv(np.ones(A.N))
    for k in (1, 3, 10, 25):
        xc, _, _, _ = oracle.cg(A, b, maxit=k, tol=0.0)
        xn, _, _, _ = oracle.cg_nb(A, b, maxit=k, tol=0.0)
        assert np.linalg.norm(xn - xc) <= 1e-10 * np.linalg.norm(xc), k


def test_cg_nb_count_and_finite_termination():
    shape = (20, 17)
    A = oracle.Operator(shape)
    b = inputs.rhs_uniform(shape, 5)
    _, itc, _, hc = oracle.cg(A, b, tol=1e-10, maxit=2000)
    x, itn, st, hn = oracle.cg_nb(A, b, tol=1e-10, maxit=2000)
    assert st == oracle.OK and abs(itn - itc) <= 1
    assert A.relres(b, x) <= 1e-10 * (1 + 1e-3)
    M = laplacian_dense((4, 4))
    distinct = len(np.unique(np.round(np.linalg.eigvalsh(M) / 8.0, 10)))
    _, it, st, _ = oracle.cg_nb(oracle.Operator((4, 4)), inputs.uniform_pm1(12, 1, 16), maxit=100, tol=1e-11)
    assert st == oracle.OK and it <= distinct


def test_cg_nb_paper_order_returns_next_iterate():
    # the printed order tests at the top of the next iteration and then
    # applies x = x_l + alpha_l p_l: the CG iterate one step further
    shape = (19, 13)
    A = oracle.Operator(shape)
    b = inputs.rhs_uniform(shape, 9)
    _, l, st, _ = oracle.cg_nb(A, b, tol=1e-8, maxit=2000)
    xp, lp, stp, _ = oracle.cg_nb(A, b, tol=1e-8, maxit=2000, paper_order=True)
    xc, _, _, _ = oracle.cg(A, b, maxit=l + 1, tol=0.0)
    assert st == stp == oracle.OK and lp == l
    assert np.linalg.norm(xp - xc) <= 1e-9 * np.linalg.norm(xc)


def test_bicgstab_b1_late_test_and_final_step():
    # B1 detects ||r_l|| <= tol inside iteration l+1 and completes that
    # iteration: the classical iterate x_{l+1} (without the half-step exit)
    shape = (14, 11)
    beta = inputs.upwind_beta(shape, 0.5)
    A = oracle.Operator(shape, oracle.UPWIND, beta)
    b = inputs.rhs_uniform(shape, 4)
    ref = np.linalg.solve(upwind_dense(shape, beta), b)
    xb, itb, stb, hb, nrb = oracle.bicgstab_b1(A, b, tol=1e-9, maxit=2000, restart_eps=0.0)
    assert stb == oracle.OK and nrb == 0
    l = itb - 1
    assert hb[l] <= 1e-9 and (l == 0 or hb[l - 1] > 1e-9)
    xc, itc, _, _, _ = oracle.bicgstab(A, b, tol=0.0, maxit=itb, restart_eps=0.0)
    assert itc == itb
    assert np.linalg.norm(xb - xc) <= 1e-10 * np.linalg.norm(xc)
    xs, _, st, _, _ = oracle.bicgstab_b1(A, b, tol=1e-13, maxit=2000)
    assert st == oracle.OK and np.linalg.norm(xs - ref) <= 1e-11 * np.linalg.norm(ref)


# --------------------------------------------------------------------------
# Adjoint gradient
# --------------------------------------------------------------------------

def _loss_dense(shape, logk, f, u_obs):
    k = np.exp(logk)
    M = oracle.Operator(shape, oracle.DIFFUSION, k=k).dense()
    u = np.linalg.solve(M, f)
    return float(np.sum((u - u_obs) ** 2)), u, M


@pytest.mark.parametrize("shape", [(4, 4, 4), (5, 3)])
def test_grad_logk_matches_dense_finite_differences(shape):
    N = int(np.prod(shape))
    logk = inputs.normal(1, inputs.STREAM_K, N, 0.5)
    f = inputs.uniform_pm1(1, 1, N)
    logk2 = inputs.normal(1, inputs.STREAM_K2, N, 0.5)
    M2 = oracle.Operator(shape, oracle.DIFFUSION, k=np.exp(logk2)).dense()
    u_obs = np.linalg.solve(M2, f)
    L0, u, M = _loss_dense(shape, logk, f, u_obs)
    lam = np.linalg.solve(M.T, 2 * (u - u_obs))
    g = oracle.grad_logk(oracle.Operator(shape, oracle.DIFFUSION, k=np.exp(logk)), u, lam)
    eps = 1e-6
    gfd = np.empty(N)
    for i in range(N):
        lp, lm = logk.copy(), logk.copy()
        lp[i] += eps
        lm[i] -= eps
        gfd[i] = (_loss_dense(shape, lp, f, u_obs)[0] - _loss_dense(shape, lm, f, u_obs)[0]) / (2 * eps)
    assert np.linalg.norm(g - gfd) <= 1e-7 * np.linalg.norm(gfd)
    # dL/df = lambda: u is linear in f, so a central difference is exact up to rounding
    for i in range(0, N, max(1, N // 7)):
        fp, fm = f.copy(), f.copy()
        fp[i] += 1e-3
        fm[i] -= 1e-3
        up, um = np.linalg.solve(M, fp), np.linalg.solve(M, fm)
        d = (np.sum((up - u_obs) ** 2) - np.sum((um - u_obs) ** 2)) / 2e-3
        assert abs(d - lam[i]) <= 1e-8 * max(1.0, np.abs(lam).max())
