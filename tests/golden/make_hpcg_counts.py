"""Writes tests/golden/hpcg_counts.json: the FP64 oracle's iteration counts on
the paper's benchmark system (section 4.1): HPCG's 7- and 27-point matrices
(diagonal 27, -1 per neighbour), b = A 1 (exact solution x = 1), x0 = 0, the
paper's absolute criterion ||r||_2 < 1e-6 (as a relative tolerance 1e-6/||b||),
BiCGStab restart threshold 1e-5, on the grid of one node of the paper's runs:
48 ranks of 128^3 along z = 128 x 128 x 6144.  Calls only the oracle.

The paper prints, for these systems on one node: 7-point BiCGStab 8, CG 12,
Gauss-Seidel 9, Jacobi 18; 27-point BiCGStab 45, CG 72, Gauss-Seidel 142,
Jacobi 515 (section 4.1).  Its Gauss-Seidel is processor-local (not the
lexicographic sweep), so only the other counts are comparable.

Run from the repository root:  python tests/golden/make_hpcg_counts.py [name ...]
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "hpcg_counts.json")
SHAPE = (128, 128, 6144)
EPS = 1e-6
PAPER = {"hpcg7": {"bicgstab": 8, "cg": 12, "jacobi": 18, "gauss_seidel_symmetric": 9},
         "hpcg27": {"bicgstab": 45, "cg": 72, "jacobi": 515, "gauss_seidel_symmetric": 142}}


def run(name):
    kind, solver = name.split(".")
    A = oracle.Operator(SHAPE, oracle.HPCG7 if kind == "hpcg7" else oracle.HPCG27)
    b = A.spmv(np.ones(A.N))
    bn = float(np.sqrt(oracle.dot(b, b)))
    tol = EPS / bn
    t0 = time.time()
    if solver == "cg":
        x, it, st, h = oracle.cg(A, b, tol=tol, maxit=5000)
    elif solver == "bicgstab":
        x, it, st, h, _ = oracle.bicgstab(A, b, tol=tol, maxit=5000, restart_eps=1e-5)
    elif solver == "jacobi":
        x, it, st, h = oracle.jacobi(A, b, tol=tol, maxit=5000)
    else:
        x, it, st, h = oracle.gauss_seidel(A, b, tol=tol, maxit=5000, mode=oracle.GS_SYMMETRIC)
    rec = {"iters": int(it), "status": int(st), "norm_b": bn, "tol_rel": tol,
           "max_err_vs_ones": float(np.max(np.abs(x - 1.0))), "cpu_seconds": round(time.time() - t0, 1)}
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    data.setdefault(kind, {})[solver] = rec
    data["grid"] = list(SHAPE)
    data["paper"] = PAPER
    data["criterion"] = "absolute ||b - A x||_2 < 1e-6 (recursive residual for CG/BiCGStab), x0 = 0, b = A 1"
    with open(OUT + ".tmp", "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(OUT + ".tmp", OUT)
    print(name, rec, flush=True)


if __name__ == "__main__":
    names = sys.argv[1:] or ["hpcg7.cg", "hpcg7.bicgstab", "hpcg7.jacobi", "hpcg7.gauss_seidel_symmetric",
                             "hpcg27.cg", "hpcg27.bicgstab", "hpcg27.jacobi"]
    for n in names:
        run(n)
