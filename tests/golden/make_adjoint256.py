"""Writes tests/golden/adjoint256_grad.json: the FP64 oracle's adjoint
gradient dL/dlog k of the 256^3 variable-diffusion workload at 64 seeded
cells, with the quantities it rests on.

Workload: -div(k grad u) = f on 256^3 interior nodes, log k ~ N(0, 0.5^2)
i.i.d. (seed 0, stream 2), f ~ U(-1, 1) (seed 0, stream 1); u_obs solves the
same f with k_obs from stream 3; L = sum_i (u_i - u_obs,i)^2.  The oracle
solves A(k) u = f, A(k_obs) u_obs = f and the adjoint A(k) lam = 2 (u - u_obs)
with its FP64 CG to the relative tolerance 1e-12, then evaluates its per-cell
gradient formula g = dL/dlog k.  Stored: the 64 cells (the first 64 distinct
draws of the finite-difference stream, inputs.distinct_cells), g there, the
2-norm of the whole g, L, the three CG iteration counts and final residuals,
and the solutions u and lam at 1024 further seeded cells with their 2-norms
(the FP64 oracle solutions the GPU's FP64 and mixed-precision solves are
compared with).

Calls only the oracle and the seeded input generator.  Run from the repository
root:  python tests/golden/make_adjoint256.py  (minutes with the OpenMP build
of the oracle, whose results are bitwise those of the sequential one).
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

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "adjoint256_grad.json")


def main():
    shape = (256, 256, 256)
    N = int(np.prod(shape))
    t0 = time.time()
    logk = inputs.log_k(shape, 0.5, 0)
    f = inputs.rhs_uniform(shape, 0)
    k = np.exp(logk)
    k_obs = np.exp(inputs.log_k(shape, 0.5, 0, inputs.STREAM_K2))
    ctx = oracle.all_cores() if oracle.have_all_cores() else contextlib.nullcontext(1)
    with ctx as threads:
        A = oracle.Operator(shape, oracle.DIFFUSION, k=k)
        A_obs = oracle.Operator(shape, oracle.DIFFUSION, k=k_obs)
        u, it_u, st_u, h_u = oracle.cg(A, f, tol=1e-12, maxit=20000)
        print("u", it_u, st_u, time.time() - t0, flush=True)
        u_obs, it_o, st_o, h_o = oracle.cg(A_obs, f, tol=1e-12, maxit=20000)
        print("u_obs", it_o, st_o, time.time() - t0, flush=True)
        d = 2.0 * (u - u_obs)
        lam, it_l, st_l, h_l = oracle.cg(A, d, tol=1e-12, maxit=20000)
        print("lam", it_l, st_l, time.time() - t0, flush=True)
        g = oracle.grad_logk(A, u, lam)
    cells = inputs.distinct_cells(N, 64)
    # the solutions themselves, sampled: the forward solution u and the adjoint
    # lam at 1024 distinct cells of a second draw (seed 1 of the same stream)
    ucells = inputs.distinct_cells(N, 1024, seed=1)
    rec = {
        "workload": ("adjoint256: 256^3 diffusion, log k ~ N(0, 0.5^2) seed 0 stream 2, f ~ U(-1,1) seed 0 "
                     "stream 1, u_obs with k_obs from stream 3, L = sum (u - u_obs)^2; oracle FP64 CG to 1e-12"),
        "cells": [int(c) for c in cells],
        "grad_at_cells": [float(v) for v in g[cells]],
        "grad_norm2": float(np.linalg.norm(g)),
        "solution_cells": [int(c) for c in ucells],
        "u_at_cells": [float(v) for v in u[ucells]],
        "lam_at_cells": [float(v) for v in lam[ucells]],
        "u_norm2": float(np.linalg.norm(u)),
        "lam_norm2": float(np.linalg.norm(lam)),
        "loss": float(np.sum((u - u_obs) ** 2)),
        "cg_iters": {"u": it_u, "u_obs": it_o, "lam": it_l},
        "cg_final_rel_res": {"u": float(h_u[-1]), "u_obs": float(h_o[-1]), "lam": float(h_l[-1])},
        "status": [st_u, st_o, st_l],
        "threads": threads,
        "cpu_seconds": round(time.time() - t0, 1),
    }
    with open(OUT + ".tmp", "w") as fo:
        json.dump(rec, fo, indent=1, sort_keys=True)
    os.replace(OUT + ".tmp", OUT)
    print(rec)


if __name__ == "__main__":
    main()
