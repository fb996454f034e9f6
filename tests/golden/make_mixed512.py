"""Writes tests/golden/mixed512_solution.json: the FP64 oracle's solution of
the 512^3 variable-diffusion workload, sampled.

Workload: -div(k grad u) = f on 512^3 interior nodes, log k ~ N(0, 1) i.i.d.
(seed 0, stream 2), f ~ U(-1, 1) (seed 0, stream 1).  The oracle solves it
with its FP64 CG from x0 = 0 to the relative residual 1e-10 (the tolerance the
GPU's FP64 CG and mixed-precision refinement are run to).  Stored: the solution
at 4096 distinct seeded cells (seed 2 of the finite-difference stream,
inputs.distinct_cells), its 2-norm, ||b||, the oracle's true relative residual
of that solution, the iteration count, and min k (the constant of the lower
bound on the operator's smallest eigenvalue the comparison uses).  The whole
solution (1 GB) is not stored.

Calls only the oracle and the seeded input generator.  Run from the
repository root:  python tests/golden/make_mixed512.py  (hours on a few cores
with the OpenMP build of the oracle, whose results are bitwise those of the
sequential one).
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

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mixed512_solution.json")


def main():
    shape = (512, 512, 512)
    N = int(np.prod(shape))
    t0 = time.time()
    k = np.exp(inputs.log_k(shape, 1.0, 0))
    b = inputs.rhs_uniform(shape, 0)
    ctx = oracle.all_cores() if oracle.have_all_cores() else contextlib.nullcontext(1)
    with ctx as threads:
        A = oracle.Operator(shape, oracle.DIFFUSION, k=k)
        x, it, st, _h = oracle.cg(A, b, tol=1e-10, maxit=20000)
        print("x", it, st, time.time() - t0, flush=True)
        rel = A.relres(b, x)
    cells = inputs.distinct_cells(N, 4096, seed=2)
    out = {
        "workload": "512^3 diffusion, log k ~ N(0, 1) (seed 0), f ~ U(-1, 1) (seed 0), oracle FP64 CG to 1e-10",
        "cells": [int(c) for c in cells],
        "x_at_cells": [float(v) for v in x[cells]],
        "x_norm2": float(np.linalg.norm(x)),
        "b_norm2": float(np.linalg.norm(b)),
        "true_rel_res": float(rel),
        "iters": int(it),
        "status": int(st),
        "k_min": float(k.min()),
        "threads": int(threads),
        "cpu_seconds": round(time.time() - t0, 1),
    }
    with open(OUT, "w") as fh:
        json.dump(out, fh)
    print({k_: v for k_, v in out.items() if k_ not in ("cells", "x_at_cells")})


if __name__ == "__main__":
    main()
