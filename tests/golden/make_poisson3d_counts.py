"""Writes tests/golden/poisson3d_256_counts.json: the FP64 oracle's iteration
counts and final relative residuals for the 3-D Poisson workload at 256^3
(CG on the 7-point Laplacian, BiCGStab on the upwind convection-diffusion
operator with beta = (1, 0.5, 0.25) scaled to cell Peclet 0.5), tolerance
1e-10 from x0 = 0, right-hand side U(-1, 1) from seed 0 (stream 1).

Besides the count of the unperturbed run, each record holds the oracle's own
spread: its counts when b is multiplied by (1 + 1e-13 z), z ~ N(0, 1) per
entry from numpy's default_rng(1234), for `reps` draws.  For BiCGStab it also
holds where the restarts of Algorithm 2 fired (the iterations after which a
restart was taken), the value sqrt|r . r'| that the restart test compared
with eps' = 1e-5 there, and the whole recursive residual history and r_k . r'
trace of the unperturbed run.

Calls only the oracle and the seeded input generator.  Run from the repository
root:  python tests/golden/make_poisson3d_counts.py [cg|bicgstab] [reps]
(the OpenMP build of the oracle is used when present: its results are
bitwise those of the sequential build).
"""
import contextlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2305_05988_gb300 import inputs  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "poisson3d_256_counts.json")


def main(which, reps):
    shape = (256, 256, 256)
    b = inputs.rhs_uniform(shape, 0)
    t0 = time.time()
    ctx = oracle.all_cores() if oracle.have_all_cores() else contextlib.nullcontext(1)
    with ctx:
        if which == "cg":
            A = oracle.Operator(shape)
            x, it, st, hist = oracle.cg(A, b, tol=1e-10, maxit=5000)
            rec = {"iters": it, "status": st, "final_rel_res": float(hist[-1]), "true_rel_res": A.relres(b, x)}
        else:
            A = oracle.Operator(shape, oracle.UPWIND, inputs.upwind_beta(shape, 0.5))
            x, it, st, hist, alpha, at = oracle.bicgstab_trace(A, b, tol=1e-10, maxit=5000, restart_eps=1e-5)
            rec = {"iters": it, "status": st, "restarts": len(at), "final_rel_res": float(hist[-1]),
                   "true_rel_res": A.relres(b, x), "restart_at": at,
                   "sqrt_abs_alpha_at_restart": [float(np.sqrt(abs(alpha[k]))) for k in at],
                   "history": [float(v) for v in hist], "alpha": [float(v) for v in alpha]}
        rec["cpu_seconds"] = round(time.time() - t0, 1)
        rng = np.random.default_rng(1234)
        counts = [it]
        for _ in range(reps):
            bb = b * (1.0 + 1e-13 * rng.standard_normal(b.size))
            if which == "cg":
                counts.append(oracle.cg(A, bb, tol=1e-10, maxit=5000)[1])
            else:
                counts.append(oracle.bicgstab(A, bb, tol=1e-10, maxit=5000, restart_eps=1e-5)[1])
            print(which, "perturbed run", len(counts) - 1, "->", counts[-1], flush=True)
        rec["spread_counts"] = counts
        rec["spread_note"] = "counts of the unperturbed run, then under b (1 + 1e-13 z), z ~ N(0,1), default_rng(1234)"
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    data[which] = rec
    data["workload"] = ("poisson3d 256^3, tol 1e-10, x0 = 0, b ~ U(-1,1) seed 0 stream 1; "
                        "bicgstab: upwind beta = (1, 0.5, 0.25)/h (cell Peclet 0.5), restart eps' = 1e-5")
    with open(OUT + ".tmp", "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(OUT + ".tmp", OUT)
    print(which, rec)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "cg", int(sys.argv[2]) if len(sys.argv) > 2 else 4)
