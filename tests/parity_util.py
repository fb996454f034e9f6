"""Shared helpers of the GPU parity tests."""
import math

import numpy as np

import oracle


def oracle_window(A_o, b, solver, it_o, tol, reps=4, **kw):
    """Iteration-count window of the oracle itself: counts under 1e-13 relative
    input noise.  Where that spread is <= 1 the count is a stable property of
    the problem and the GPU must match it to +-2; otherwise the count depends on
    the rounding of every inner product (strong coefficient contrast: the window
    widens by the spread and 1 %; BiCGStab restarts: by the spread and 10 %)."""
    rng = np.random.default_rng(1234)
    counts = [it_o]
    restarted = False
    for q in range(reps + 1):
        bb = b if q == 0 else b * (1.0 + 1e-13 * rng.standard_normal(b.size))
        if solver == "cg":
            if q:
                counts.append(oracle.cg(A_o, bb, tol=tol, maxit=20000)[1])
        else:
            _, it, _, _, nr = oracle.bicgstab(A_o, bb, tol=tol, maxit=20000, **kw)
            restarted |= nr > 0
            if q:
                counts.append(it)
    lo, hi = min(counts), max(counts)
    if hi - lo <= 1 and not restarted:
        return it_o - 2, it_o + 2, counts
    # BiCGStab restarts on an absolute threshold of |r . r'|; when they fire,
    # where they fire depends on the rounding of every inner product (on the
    # 128^2 Laplacian the oracle alone ranges 680-756 iterations under 1-ulp
    # perturbations of b, about 10 %)
    frac = 0.10 if restarted else 0.01
    slack = 2 + int(math.ceil(frac * it_o))
    return lo - slack, hi + slack, counts


