"""Shared helpers of the GPU parity tests."""
import math

import numpy as np

import oracle


def oracle_window(A_o, b, solver, it_o, tol, reps=4, **kw):
    """Iteration-count window of the oracle itself: counts under 1e-13 relative
    input noise.  Where that spread is <= 1 the count is a stable property of
    the problem and the GPU must match it to +-2; otherwise the count depends on
    the rounding of every inner product (BiCGStab's restart rule, strong
    coefficient contrast) and the window widens by the spread and 1 %."""
    rng = np.random.default_rng(1234)
    counts = [it_o]
    for _ in range(reps):
        bb = b * (1.0 + 1e-13 * rng.standard_normal(b.size))
        if solver == "cg":
            counts.append(oracle.cg(A_o, bb, tol=tol, maxit=20000)[1])
        else:
            counts.append(oracle.bicgstab(A_o, bb, tol=tol, maxit=20000, **kw)[1])
    lo, hi = min(counts), max(counts)
    if hi - lo <= 1:
        return it_o - 2, it_o + 2, counts
    slack = 2 + int(math.ceil(0.01 * it_o))
    return lo - slack, hi + slack, counts


