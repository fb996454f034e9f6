"""Independent dense constructions used to pin the oracle (test helpers).

These do not call the oracle.  The constant-coefficient operators are built as
Kronecker sums of 1-D tridiagonal matrices (storage order i fastest, so the
factor acting along x is the last Kronecker factor); the closed-form
eigenpairs are the textbook ones for tridiagonal Toeplitz matrices.
"""
import math

import numpy as np


def tridiag(n, lower, diag, upper):
    T = np.zeros((n, n))
    for i in range(n):
        T[i, i] = diag
        if i > 0:
            T[i, i - 1] = lower
        if i < n - 1:
            T[i, i + 1] = upper
    return T


def kron_sum(mats):
    """sum_d I x .. x T_d x .. x I with mats given in (x, y, z) order, x fastest."""
    mats = list(mats)
    sizes = [m.shape[0] for m in mats]
    N = int(np.prod(sizes))
    A = np.zeros((N, N))
    for d, T in enumerate(mats):
        # factors listed slowest-first: z, y, x
        factors = []
        for e in reversed(range(len(mats))):
            factors.append(T if e == d else np.eye(sizes[e]))
        K = factors[0]
        for F in factors[1:]:
            K = np.kron(K, F)
        A += K
    return A


def laplacian_dense(shape):
    mats = []
    for n in shape:
        h = 1.0 / (n + 1)
        mats.append(tridiag(n, -1.0 / h**2, 2.0 / h**2, -1.0 / h**2))
    return kron_sum(mats)


def upwind_dense(shape, beta):
    mats = []
    for d, n in enumerate(shape):
        h = 1.0 / (n + 1)
        b = beta[d]
        mats.append(tridiag(n, -1.0 / h**2 - b / h, 2.0 / h**2 + b / h, -1.0 / h**2))
    return kron_sum(mats)


def toeplitz_eig_1d(n, lower, diag, upper, m):
    """Eigenpair m (1..n) of tridiag(lower, diag, upper): requires lower*upper > 0."""
    theta = m * math.pi / (n + 1)
    rho = math.sqrt(lower / upper)
    i = np.arange(1, n + 1)
    v = rho**i * np.sin(i * theta)
    lam = diag + 2.0 * math.copysign(math.sqrt(lower * upper), upper) * math.cos(theta)
    return lam, v


def tensor_vec(vs):
    """Outer product of 1-D vectors given in (x, y, z) order, flattened x fastest."""
    out = vs[-1]
    for v in reversed(vs[:-1]):
        out = np.multiply.outer(out, v)
    return out.reshape(-1)


def grid_coords(shape):
    """Interior node coordinates ((i+1) h_x, ...) as arrays flattened x fastest."""
    axes = [(np.arange(n) + 1.0) / (n + 1) for n in shape]
    mesh = np.meshgrid(*reversed(axes), indexing="ij")  # z, y, x order
    return [m.reshape(-1) for m in reversed(mesh)]
