"""FP64 CPU oracle for the structured-grid iterative solvers (test infrastructure).

This package is test infrastructure, not part of the product.  Only the test
suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it.  It shares no code with the CUDA library and never calls it.

The arithmetic lives in ``oracle.c`` (plain sequential C, compiled with
``-O2 -ffp-contract=off``); this module only compiles it with gcc and marshals
numpy arrays through ctypes.  Which passage of the paper each routine follows
is stated beside it in ``oracle.c``:

* operators and SpMV      -- problem statement A x = b, section 3.1 / 4.1
* Jacobi, Gauss-Seidel    -- section 3.1 (symmetric GS = forward + backward)
* CG                      -- classical CG of HPCCG, section 3.2
* BiCGStab                -- Algorithm 2's normalised shadow residual and
                             restart rule, classical statement order
* adjoint gradient        -- dL/dlog k of the diffusion operator (not in the
                             paper; derived from A(k) u = f)
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_OMP_PATH = os.path.join(_BUILD, "liboracle_omp.so")
_lock = threading.Lock()
_libs = {}
_use_omp = False

LAPLACIAN, UPWIND, DIFFUSION, HPCG7, HPCG27 = 0, 1, 2, 3, 4
GS_FORWARD, GS_BACKWARD, GS_SYMMETRIC = 0, 1, 2
OK, NOT_CONVERGED, BREAKDOWN = 0, 1, -3


def _compile(out: str, extra, force: bool) -> str:
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"] + list(extra) + \
        ["-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, plain C11, sequential:
    the parity checker) and, where gcc has OpenMP, _build/liboracle_omp.so
    (the same source with its element-wise loops on all host cores; bitwise
    the same results, used only to time the oracle and to run long
    reference solves)."""
    path = _compile(_LIB_PATH, [], force)
    try:
        _compile(_OMP_PATH, ["-fopenmp"], force)
    except (subprocess.CalledProcessError, OSError):
        pass
    return path


class _Op(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("kind", ctypes.c_int),
                ("n", ctypes.c_int64 * 3), ("h", ctypes.c_double * 3),
                ("beta", ctypes.c_double * 3), ("k", ctypes.c_void_p)]


def _declare(lib):
    if True:
        if True:
            P = ctypes.POINTER
            dp = ctypes.c_void_p
            op = P(_Op)
            lib.ora_size.argtypes = [op]; lib.ora_size.restype = ctypes.c_int64
            lib.ora_spmv.argtypes = [op, dp, dp]; lib.ora_spmv.restype = None
            lib.ora_dense.argtypes = [op, dp, ctypes.c_int64]; lib.ora_dense.restype = ctypes.c_int
            lib.ora_relres.argtypes = [op, dp, dp]; lib.ora_relres.restype = ctypes.c_double
            lib.ora_dot.argtypes = [ctypes.c_int64, dp, dp]; lib.ora_dot.restype = ctypes.c_double
            lib.ora_jacobi.argtypes = [op, dp, dp, ctypes.c_int, ctypes.c_double, dp, P(ctypes.c_int)]
            lib.ora_jacobi.restype = ctypes.c_int
            lib.ora_gs_sweep.argtypes = [op, dp, dp, ctypes.c_int]; lib.ora_gs_sweep.restype = None
            lib.ora_gauss_seidel.argtypes = [op, dp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                             dp, P(ctypes.c_int)]
            lib.ora_gauss_seidel.restype = ctypes.c_int
            lib.ora_cg.argtypes = [op, dp, dp, ctypes.c_int, ctypes.c_double, dp, P(ctypes.c_int)]
            lib.ora_cg.restype = ctypes.c_int
            lib.ora_bicgstab.argtypes = [op, dp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                         dp, P(ctypes.c_int), P(ctypes.c_int), dp, dp]
            lib.ora_bicgstab.restype = ctypes.c_int
            lib.ora_cg_nb.argtypes = [op, dp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_int, dp,
                                      P(ctypes.c_int)]
            lib.ora_cg_nb.restype = ctypes.c_int
            lib.ora_bicgstab_b1.argtypes = [op, dp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                            dp, P(ctypes.c_int), P(ctypes.c_int)]
            lib.ora_bicgstab_b1.restype = ctypes.c_int
            lib.ora_grad_logk.argtypes = [op, dp, dp, dp]; lib.ora_grad_logk.restype = ctypes.c_int
            lib.ora_set_threads.argtypes = [ctypes.c_int]; lib.ora_set_threads.restype = None
            lib.ora_threads.argtypes = []; lib.ora_threads.restype = ctypes.c_int
    return lib


def _load():
    """The sequential build, or the OpenMP build inside ``all_cores()``."""
    key = "omp" if _use_omp else "seq"
    with _lock:
        lib = _libs.get(key)
        if lib is None:
            path = build()
            if key == "omp":
                if not os.path.exists(_OMP_PATH):
                    raise RuntimeError("the OpenMP build of the oracle is not available (gcc without -fopenmp)")
                path = _OMP_PATH
            lib = _libs[key] = _declare(ctypes.CDLL(path))
    return lib


def have_all_cores() -> bool:
    """True when the OpenMP build of the oracle exists."""
    build()
    return os.path.exists(_OMP_PATH)


@contextlib.contextmanager
def all_cores(threads: int = 0):
    """Run the oracle calls inside the block on the OpenMP build: element-wise
    loops (SpMV, residuals, vector updates, Jacobi sweeps, the gradient) on
    ``threads`` host threads (0 = all cores this process may use), inner
    products and Gauss-Seidel sweeps sequential.  Results are bitwise those of
    the sequential build.  Yields the thread count in use."""
    global _use_omp
    prev = _use_omp
    _use_omp = True
    try:
        lib = _load()
        n = threads if threads > 0 else len(os.sched_getaffinity(0))
        lib.ora_set_threads(int(n))
        yield lib.ora_threads()
    finally:
        _use_omp = prev


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class Operator:
    """A structured-grid operator: shape (n_x[, n_y[, n_z]]), kind and parameters.

    ``k`` (diffusion only) is the per-cell coefficient in lexicographic order
    (i fastest); it is copied and kept alive by this object.
    """

    def __init__(self, shape, kind=LAPLACIAN, beta=(0.0, 0.0, 0.0), k=None):
        shape = tuple(int(s) for s in shape)
        if not 1 <= len(shape) <= 3 or min(shape) < 1:
            raise ValueError("bad grid shape %r" % (shape,))
        self.shape = shape
        self.kind = kind
        self.beta = tuple(float(b) for b in beta) + (0.0,) * (3 - len(beta))
        self.N = int(np.prod(shape))
        self._k = None
        if kind == DIFFUSION:
            if k is None:
                raise ValueError("diffusion operator needs k")
            self._k = _f64(k).reshape(-1).copy()
            if self._k.size != self.N:
                raise ValueError("k has wrong size")
        s = _Op()
        s.ndim = len(shape)
        s.kind = kind
        for d in range(3):
            s.n[d] = shape[d] if d < len(shape) else 1
            s.h[d] = 1.0 / (s.n[d] + 1) if d < len(shape) else 1.0
            s.beta[d] = self.beta[d]
        s.k = self._k.ctypes.data if self._k is not None else None
        self._s = s

    @property
    def h(self):
        return tuple(1.0 / (n + 1) for n in self.shape)

    @property
    def k(self):
        return self._k

    def _ref(self):
        return ctypes.byref(self._s)

    def spmv(self, x):
        x = _f64(x).reshape(-1)
        assert x.size == self.N
        y = np.empty(self.N)
        _load().ora_spmv(self._ref(), _ptr(x), _ptr(y))
        return y

    def dense(self, maxN=4096):
        if self.N > maxN:
            raise ValueError("grid too large for dense assembly")
        M = np.empty((self.N, self.N))
        rc = _load().ora_dense(self._ref(), _ptr(M), maxN)
        assert rc == 0
        return M

    def relres(self, b, x):
        b = _f64(b).reshape(-1); x = _f64(x).reshape(-1)
        return _load().ora_relres(self._ref(), _ptr(b), _ptr(x))


def dot(a, b):
    """Inner product of two vectors (compensated summation in index order)."""
    a = _f64(a).reshape(-1); b = _f64(b).reshape(-1)
    assert a.size == b.size
    return _load().ora_dot(a.size, _ptr(a), _ptr(b))


def _hist(maxit, want):
    return np.full(maxit + 1, np.nan) if want else None


def jacobi(A: Operator, b, x0=None, maxit=100, tol=0.0, history=False):
    """Jacobi sweeps; returns (x, iters, status, hist)."""
    b = _f64(b).reshape(-1)
    x = np.zeros(A.N) if x0 is None else _f64(x0).reshape(-1).copy()
    h = _hist(maxit, history)
    it = ctypes.c_int(0)
    st = _load().ora_jacobi(A._ref(), _ptr(b), _ptr(x), int(maxit), float(tol),
                            _ptr(h) if h is not None else None, ctypes.byref(it))
    return x, it.value, st, (h[: it.value + 1] if h is not None and tol > 0 else None)


def gauss_seidel(A: Operator, b, x0=None, maxit=100, tol=0.0, mode=GS_FORWARD, history=False):
    """Gauss-Seidel sweeps (mode forward / backward / symmetric); returns (x, iters, status, hist)."""
    b = _f64(b).reshape(-1)
    x = np.zeros(A.N) if x0 is None else _f64(x0).reshape(-1).copy()
    h = _hist(maxit, history)
    it = ctypes.c_int(0)
    st = _load().ora_gauss_seidel(A._ref(), _ptr(b), _ptr(x), int(maxit), float(tol), int(mode),
                                  _ptr(h) if h is not None else None, ctypes.byref(it))
    return x, it.value, st, (h[: it.value + 1] if h is not None and tol > 0 else None)


def gs_sweep(A: Operator, b, x, backward=False):
    """One in-place Gauss-Seidel sweep on a copy of x; returns the new x."""
    b = _f64(b).reshape(-1)
    x = _f64(x).reshape(-1).copy()
    _load().ora_gs_sweep(A._ref(), _ptr(b), _ptr(x), int(bool(backward)))
    return x


def cg(A: Operator, b, x0=None, maxit=1000, tol=1e-10):
    """Classical CG; returns (x, iters, status, hist)."""
    b = _f64(b).reshape(-1)
    x = np.zeros(A.N) if x0 is None else _f64(x0).reshape(-1).copy()
    h = _hist(maxit, True)
    it = ctypes.c_int(0)
    st = _load().ora_cg(A._ref(), _ptr(b), _ptr(x), int(maxit), float(tol), _ptr(h), ctypes.byref(it))
    return x, it.value, st, h[: it.value + 1]


def bicgstab(A: Operator, b, x0=None, maxit=1000, tol=1e-10, restart_eps=1e-5):
    """BiCGStab with restart; returns (x, iters, status, hist, restarts)."""
    b = _f64(b).reshape(-1)
    x = np.zeros(A.N) if x0 is None else _f64(x0).reshape(-1).copy()
    h = _hist(maxit, True)
    it = ctypes.c_int(0)
    nr = ctypes.c_int(0)
    st = _load().ora_bicgstab(A._ref(), _ptr(b), _ptr(x), int(maxit), float(tol), float(restart_eps),
                              _ptr(h), ctypes.byref(it), ctypes.byref(nr), None, None)
    return x, it.value, st, h[: it.value + 1], nr.value


def bicgstab_trace(A: Operator, b, x0=None, maxit=1000, tol=1e-10, restart_eps=1e-5):
    """BiCGStab as ``bicgstab`` that also returns what decides its restarts:
    (x, iters, status, hist, alpha, restart_at) with alpha[k] = r_k . r' after
    iteration k (the value the restart test compares, alpha[0] = r_0 . r') and
    restart_at the iterations after which a restart was taken."""
    b = _f64(b).reshape(-1)
    x = np.zeros(A.N) if x0 is None else _f64(x0).reshape(-1).copy()
    h = _hist(maxit, True)
    tr = np.full(maxit + 1, np.nan)
    at = np.zeros(max(maxit, 1), dtype=np.int32)
    it = ctypes.c_int(0)
    nr = ctypes.c_int(0)
    st = _load().ora_bicgstab(A._ref(), _ptr(b), _ptr(x), int(maxit), float(tol), float(restart_eps),
                              _ptr(h), ctypes.byref(it), ctypes.byref(nr), _ptr(tr), _ptr(at))
    return x, it.value, st, h[: it.value + 1], tr[: it.value + 1], [int(v) for v in at[: nr.value]]


def cg_nb(A: Operator, b, x0=None, maxit=1000, tol=1e-10, paper_order=False):
    """CG-NB (Algorithm 1); returns (x, iters, status, hist)."""
    b = _f64(b).reshape(-1)
    x = np.zeros(A.N) if x0 is None else _f64(x0).reshape(-1).copy()
    h = _hist(maxit, True)
    it = ctypes.c_int(0)
    st = _load().ora_cg_nb(A._ref(), _ptr(b), _ptr(x), int(maxit), float(tol), int(bool(paper_order)), _ptr(h),
                           ctypes.byref(it))
    return x, it.value, st, h[: it.value + 1]


def bicgstab_b1(A: Operator, b, x0=None, maxit=1000, tol=1e-10, restart_eps=1e-5):
    """BiCGStab in the statement order of Algorithm 2 (late test, final step);
    returns (x, iters, status, hist, restarts)."""
    b = _f64(b).reshape(-1)
    x = np.zeros(A.N) if x0 is None else _f64(x0).reshape(-1).copy()
    h = _hist(maxit, True)
    it = ctypes.c_int(0)
    nr = ctypes.c_int(0)
    st = _load().ora_bicgstab_b1(A._ref(), _ptr(b), _ptr(x), int(maxit), float(tol), float(restart_eps),
                                 _ptr(h), ctypes.byref(it), ctypes.byref(nr))
    return x, it.value, st, h[: it.value + 1], nr.value


def grad_logk(A: Operator, u, lam):
    """dL/dlog k per cell from the forward solution u and the adjoint lam."""
    u = _f64(u).reshape(-1); lam = _f64(lam).reshape(-1)
    g = np.empty(A.N)
    rc = _load().ora_grad_logk(A._ref(), _ptr(u), _ptr(lam), _ptr(g))
    if rc != 0:
        raise ValueError("grad_logk needs a diffusion operator")
    return g
