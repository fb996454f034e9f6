"""Seeded synthetic inputs for the structured-grid solvers.

This module holds no solver arithmetic: it only draws the right-hand sides,
diffusion coefficients and batch descriptions that both the CUDA path and the
CPU oracle consume, so that both sides see bit-identical inputs.

Generator: counter-based SplitMix64.  Value ``i`` of stream ``s`` under seed
``seed`` is ``mix64(base(seed, s) + (i + 1) * GAMMA)`` with
``base(seed, s) = mix64(seed * GAMMA + s)`` and ``mix64`` the SplitMix64
output finaliser (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014).  A uniform double in [0, 1) is the top 53 bits
times 2**-53 (exact).  Normal draws use the Box-Muller transform on two
uniforms (indices 2i and 2i+1 of the stream); they go through the platform's
``log``/``cos``, so they may differ in the last bit between machines -- both
sides of a parity test always draw them on the same machine.

Streams: 1 = right-hand side, 2 = diffusion coefficient k, 3 = second
coefficient k_obs / finite-difference cell picks, 4 = batch draws,
0x10000 + s = right-hand side of batch system s.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

STREAM_RHS = 1
STREAM_K = 2
STREAM_K2 = 3
STREAM_BATCH = 4
STREAM_FD = 5
STREAM_BATCH_RHS = 0x10000


def _mix64(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _base(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * GAMMA + np.uint64(stream & 0xFFFFFFFFFFFFFFFF)
    return _mix64(s)


def raw_u64(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Raw 64-bit draws offset .. offset+n-1 of a stream."""
    i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(_base(seed, stream) + i * GAMMA)


def uniform(seed: int, stream: int, n: int, offset: int = 0, chunk: int = 1 << 24) -> np.ndarray:
    """U[0, 1) doubles (53-bit, exact)."""
    out = np.empty(n, dtype=np.float64)
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        out[s:s + m] = (raw_u64(seed, stream, m, offset + s) >> np.uint64(11)).astype(np.float64)
    out *= 2.0 ** -53
    return out


def uniform_pm1(seed: int, stream: int, n: int) -> np.ndarray:
    """U[-1, 1) doubles: 2u - 1 (exact)."""
    u = uniform(seed, stream, n)
    u *= 2.0
    u -= 1.0
    return u


def normal(seed: int, stream: int, n: int, sigma: float = 1.0) -> np.ndarray:
    """N(0, sigma^2) doubles by Box-Muller on uniform pairs (2i, 2i+1)."""
    out = np.empty(n, dtype=np.float64)
    chunk = 1 << 23
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        u = uniform(seed, stream, 2 * m, offset=2 * s)
        u1 = 1.0 - u[0::2]                # (0, 1]
        u2 = u[1::2]
        out[s:s + m] = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)
    if sigma != 1.0:
        out *= sigma
    return out


def rhs_uniform(shape, seed: int = 0, stream: int = STREAM_RHS) -> np.ndarray:
    """Right-hand side f_i ~ U(-1, 1) on the interior nodes, lexicographic (i fastest)."""
    return uniform_pm1(seed, stream, int(np.prod(shape)))


def rhs_manufactured_2d(shape) -> np.ndarray:
    """f = 2 pi^2 sin(pi x) sin(pi y) at the interior nodes x_i = (i+1) h_x, y_j = (j+1) h_y."""
    nx, ny = shape
    x = (np.arange(nx) + 1.0) / (nx + 1)
    y = (np.arange(ny) + 1.0) / (ny + 1)
    f = 2.0 * math.pi ** 2 * np.outer(np.sin(math.pi * y), np.sin(math.pi * x))  # [j, i]
    return f.reshape(-1)


def log_k(shape, sigma: float, seed: int = 0, stream: int = STREAM_K) -> np.ndarray:
    """log k ~ N(0, sigma^2), i.i.d. per cell."""
    return normal(seed, stream, int(np.prod(shape)), sigma)


@dataclass(frozen=True)
class BatchSystem:
    index: int
    shape: tuple
    solver: str          # "cg" (symmetric diffusion, k = 1) or "bicgstab" (upwind)
    peclet: float        # cell Peclet number (upwind systems only)

    @property
    def N(self) -> int:
        return int(np.prod(self.shape))


def batch_systems(nsys: int = 512, seed: int = 0, side_min: int = 16, side_max: int = 256):
    """Describe a batch of independent systems.

    System s draws three uniforms (3s, 3s+1, 3s+2) from the batch stream:
    side = round(side_min * (side_max/side_min)**U), dim = 2 if U' < 0.5 else 3,
    Peclet = 0.1 + 0.9 U''.  Even s -> CG on the symmetric (k = 1) diffusion
    operator, odd s -> BiCGStab on the upwind convection-diffusion operator.
    """
    u = uniform(seed, STREAM_BATCH, 3 * nsys)
    out = []
    ratio = side_max / side_min
    for s in range(nsys):
        side = int(round(side_min * ratio ** u[3 * s]))
        dim = 2 if u[3 * s + 1] < 0.5 else 3
        pe = 0.1 + 0.9 * u[3 * s + 2]
        out.append(BatchSystem(s, (side,) * dim, "cg" if s % 2 == 0 else "bicgstab", float(pe)))
    return out


def upwind_beta(shape, peclet: float = 0.5, direction=(1.0, 0.5, 0.25)):
    """Velocity beta = direction scaled so that the cell Peclet number max_d beta_d h_d / 2 equals peclet."""
    nd = len(shape)
    h = [1.0 / (n + 1) for n in shape]
    d = list(direction[:nd])
    m = max(d[i] * h[i] for i in range(nd))
    scale = 2.0 * peclet / m
    return tuple(d[i] * scale for i in range(nd)) + (0.0,) * (3 - nd)


def distinct_cells(N: int, count: int, seed: int = 0, stream: int = STREAM_FD) -> np.ndarray:
    """`count` distinct cell indices in [0, N): floor(U N) for the stream's
    uniforms in draw order, repeats skipped (the finite-difference cells of the
    adjoint check)."""
    if count > N:
        raise ValueError("more cells than the grid holds")
    out, seen, off = [], set(), 0
    while len(out) < count:
        u = uniform(seed, stream, 4 * count, offset=off)
        off += 4 * count
        for c in (u * N).astype(np.int64):
            if int(c) not in seen:
                seen.add(int(c))
                out.append(int(c))
                if len(out) == count:
                    break
    return np.array(out, dtype=np.int64)
