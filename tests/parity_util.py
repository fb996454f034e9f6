"""Shared helpers of the GPU parity tests."""
import numpy as np

import oracle


def maxrel(a, ref):
    """Element-wise error scaled by the largest reference entry:
    max_i |a_i - ref_i| / max_i |ref_i| (0 / 0 = 0).  Beside a relative 2-norm
    it catches a single wrong entry (a tile edge, a halo node) that the norm
    of a long vector would average away."""
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    ref = np.asarray(ref, dtype=np.float64).reshape(-1)
    scale = np.max(np.abs(ref)) if ref.size else 0.0
    err = np.max(np.abs(a - ref)) if ref.size else 0.0
    return err / scale if scale > 0 else err


def oracle_spread(A_o, b, solver, it_o, x_o, tol, reps=8, **kw):
    """The oracle's own sensitivity to rounding-level changes of its input.

    solver: "cg", "bicgstab" or "bicgstab_b1" (Algorithm 2's order).  Runs the
    oracle `reps` more times with b multiplied entry-wise by
    (1 + 1e-13 z), z ~ N(0, 1) (numpy default_rng(1234)), and returns
    (counts, restarted, xdev): the iteration counts (the unperturbed one
    first), whether any run restarted (BiCGStab), and the largest relative
    2-norm distance between a perturbed run's iterate after exactly it_o
    iterations and the unperturbed x_o.  A GPU solve differs from the oracle
    only in rounding order, which perturbs the iteration at least as much as a
    1e-13 change of b does, so this spread is the scale of disagreement that
    the oracle itself shows between equally valid runs."""
    rng = np.random.default_rng(1234)
    counts = [it_o]
    restarted = False
    xdev = 0.0
    if solver in ("bicgstab", "bicgstab_b1"):
        run = oracle.bicgstab_b1 if solver == "bicgstab_b1" else oracle.bicgstab
        restarted = run(A_o, b, tol=tol, maxit=20000, **kw)[4] > 0
    nx = np.linalg.norm(x_o)
    for _ in range(reps):
        bb = b * (1.0 + 1e-13 * rng.standard_normal(b.size))
        if solver == "cg":
            counts.append(oracle.cg(A_o, bb, tol=tol, maxit=20000)[1])
            xq = oracle.cg(A_o, bb, tol=0.0, maxit=it_o)[0]
        else:
            run = oracle.bicgstab_b1 if solver == "bicgstab_b1" else oracle.bicgstab
            _, it, _, _, nr = run(A_o, bb, tol=tol, maxit=20000, **kw)
            restarted |= nr > 0
            counts.append(it)
            xq = run(A_o, bb, tol=0.0, maxit=it_o, **kw)[0]
        xdev = max(xdev, float(np.linalg.norm(xq - x_o) / nx) if nx > 0 else 0.0)
    return counts, restarted, xdev


def oracle_window(A_o, b, solver, it_o, tol, reps=8, x_o=None, **kw):
    """Iteration-count window: the oracle's count +-2 where its own count is
    stable under 1e-13 relative input noise (spread <= 1, no BiCGStab
    restart); otherwise the oracle's measured spread (min .. max over `reps`
    perturbed runs and the unperturbed one) widened by 2 on each side, the
    same +-2 applied to the range of counts the oracle itself produces.
    Returns (lo, hi, counts, stable, xdev) with xdev as in oracle_spread."""
    if x_o is None:
        if solver == "cg":
            x_o = oracle.cg(A_o, b, tol=0.0, maxit=it_o)[0]
        elif solver == "bicgstab_b1":
            x_o = oracle.bicgstab_b1(A_o, b, tol=0.0, maxit=it_o, **kw)[0]
        else:
            x_o = oracle.bicgstab(A_o, b, tol=0.0, maxit=it_o, **kw)[0]
    counts, restarted, xdev = oracle_spread(A_o, b, solver, it_o, x_o, tol, reps=reps, **kw)
    lo, hi = min(counts), max(counts)
    stable = hi - lo <= 1 and not restarted
    if stable:
        return it_o - 2, it_o + 2, counts, True, xdev
    return lo - 2, hi + 2, counts, False, xdev


def oracle_xdev(A_o, b, solver, k, x_o, reps=8, **kw):
    """Only the iterate part of oracle_spread: the largest relative distance
    between the oracle's iterate after exactly k iterations on a perturbed b
    (the same perturbations) and x_o."""
    rng = np.random.default_rng(1234)
    run = {"cg": oracle.cg, "bicgstab": oracle.bicgstab, "bicgstab_b1": oracle.bicgstab_b1}[solver]
    nx = np.linalg.norm(x_o)
    xdev = 0.0
    for _ in range(reps):
        bb = b * (1.0 + 1e-13 * rng.standard_normal(b.size))
        xq = run(A_o, bb, tol=0.0, maxit=k, **kw)[0]
        xdev = max(xdev, float(np.linalg.norm(xq - x_o) / nx) if nx > 0 else 0.0)
    return xdev


def iterate_bar(stable, xdev):
    """Tolerance for the GPU iterate against the oracle's after the same
    number of iterations: 1e-8 relative where the oracle's count is stable,
    else the larger of 1e-8 and ten times the distance the oracle's own
    perturbed runs show after that many iterations (the GPU's rounding order
    is a perturbation of the same kind; ten gives room for it being a few
    times stronger than one 1e-13 change of b)."""
    return 1e-8 if stable else max(1e-8, 10.0 * xdev)
