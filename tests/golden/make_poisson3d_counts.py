"""Writes tests/golden/poisson3d_256_counts.json: the FP64 oracle's iteration
counts and final relative residuals for the 3-D Poisson workload at 256^3
(CG on the 7-point Laplacian, BiCGStab on the upwind convection-diffusion
operator with beta = (1, 0.5, 0.25) scaled to cell Peclet 0.5), tolerance
1e-10 from x0 = 0, right-hand side U(-1, 1) from seed 0 (stream 1).

Calls only the oracle and the seeded input generator.  Run from the repository
root:  python tests/golden/make_poisson3d_counts.py [cg|bicgstab]
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2305_05988_gb300 import inputs  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "poisson3d_256_counts.json")


def main(which):
    shape = (256, 256, 256)
    b = inputs.rhs_uniform(shape, 0)
    t0 = time.time()
    if which == "cg":
        A = oracle.Operator(shape)
        x, it, st, hist = oracle.cg(A, b, tol=1e-10, maxit=5000)
        rec = {"iters": it, "status": st, "final_rel_res": float(hist[-1]), "true_rel_res": A.relres(b, x)}
    else:
        A = oracle.Operator(shape, oracle.UPWIND, inputs.upwind_beta(shape, 0.5))
        x, it, st, hist, nr = oracle.bicgstab(A, b, tol=1e-10, maxit=5000, restart_eps=1e-5)
        rec = {"iters": it, "status": st, "restarts": nr, "final_rel_res": float(hist[-1]),
               "true_rel_res": A.relres(b, x)}
    rec["cpu_seconds"] = round(time.time() - t0, 1)
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
    main(sys.argv[1] if len(sys.argv) > 1 else "cg")
