"""Python front end of libhsolve: structured-grid operators and the four
classical iterative methods of arXiv 2305.05988 (Jacobi, Gauss-Seidel, CG,
BiCGStab), running in hand-written CUDA kernels for sm_103a.

PyTorch only supplies device memory and the current CUDA stream; every step
of every solve runs inside libhsolve.  Vectors are contiguous CUDA tensors
of float64 (or float32) in lexicographic order (x fastest), i.e. a tensor of
shape (n_z, n_y, n_x) flattened.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib
from ._lib import check

_DT = {torch.float64: _lib.HS_F64, torch.float32: _lib.HS_F32}
_GS_MODES = {"forward": _lib.HS_GS_FORWARD, "backward": _lib.HS_GS_BACKWARD, "symmetric": _lib.HS_GS_SYMMETRIC}


@dataclass
class SolveInfo:
    """Outcome of a solve (mirrors hs_result)."""
    iters: int
    status: str
    status_code: int
    rel_res: float
    true_rel_res: float
    restarts: int = 0
    history: Optional[np.ndarray] = None
    outer: int = 0
    inner_iters: int = 0
    alpha_trace: Optional[np.ndarray] = None      # BiCGStab: r_k . r' per iteration (trace=True)
    restart_iters: Optional[list] = None          # BiCGStab: iterations followed by a restart

    @property
    def converged(self) -> bool:
        return self.status_code == _lib.HS_OK


class Operator:
    """A matrix-free structured-grid operator (Laplacian, upwind convection-diffusion,
    variable-coefficient diffusion, or the HPCG 7/27-point benchmark matrix) on
    n_x [* n_y [* n_z]] interior nodes with homogeneous Dirichlet boundaries and
    spacing h_d = 1/(n_d + 1) (the HPCG matrices are unscaled)."""

    def __init__(self, shape: Sequence[int], kind: str = "laplacian", beta=None, k: Optional[torch.Tensor] = None):
        lib = _lib.load()
        self.shape = tuple(int(s) for s in shape)
        self.ndim = len(self.shape)
        self.kind = kind
        self.N = int(np.prod(self.shape))
        self._grid = ctypes.c_void_p()
        self._op = ctypes.c_void_p()
        self._k = None
        n = (ctypes.c_int64 * 3)(*(list(self.shape) + [1] * (3 - self.ndim)))
        check(lib.hs_grid_create(self.ndim, n, ctypes.byref(self._grid)), "hs_grid_create")
        try:
            if kind == "laplacian":
                check(lib.hs_op_laplacian(self._grid, ctypes.byref(self._op)), "hs_op_laplacian")
            elif kind == "upwind":
                b = (ctypes.c_double * 3)(*(list(beta) + [0.0] * (3 - len(beta))))
                self.beta = tuple(float(v) for v in beta)
                check(lib.hs_op_convdiff_upwind(self._grid, b, ctypes.byref(self._op)), "hs_op_convdiff_upwind")
            elif kind == "diffusion":
                if k is None or not k.is_cuda:
                    raise ValueError("diffusion operator needs k as a CUDA tensor")
                if k.numel() != self.N or k.dtype not in _DT:
                    raise ValueError("k must hold N float64/float32 values")
                self._k = k.contiguous()
                check(lib.hs_op_diffusion(self._grid, _DT[self._k.dtype], ctypes.c_void_p(self._k.data_ptr()),
                                          ctypes.byref(self._op)), "hs_op_diffusion")
            elif kind in ("hpcg7", "hpcg27"):
                check(lib.hs_op_hpcg(self._grid, 7 if kind == "hpcg7" else 27, ctypes.byref(self._op)), "hs_op_hpcg")
            else:
                raise ValueError("unknown operator kind %r" % kind)
        finally:
            lib.hs_grid_destroy(self._grid)
            self._grid = None
        self._ws = {}

    # -- constructors -------------------------------------------------------
    @classmethod
    def laplacian(cls, shape):
        return cls(shape, "laplacian")

    @classmethod
    def upwind(cls, shape, beta):
        return cls(shape, "upwind", beta=beta)

    @classmethod
    def diffusion(cls, shape, k: torch.Tensor):
        return cls(shape, "diffusion", k=k)

    @classmethod
    def hpcg(cls, shape, points: int = 27):
        """The paper's benchmark system (section 4.1): diagonal 27, -1 for each
        of the 6 face (points=7) or 26 box (points=27) neighbours, unscaled."""
        if points not in (7, 27):
            raise ValueError("points must be 7 or 27")
        return cls(shape, "hpcg%d" % points)

    def __del__(self):
        try:
            if getattr(self, "_op", None) is not None and self._op.value:
                _lib.load().hs_op_destroy(self._op)
                self._op = None
        except Exception:
            pass

    # -- helpers ----------------------------------------------------------------
    def _vec(self, t: torch.Tensor, name: str) -> torch.Tensor:
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError("%s must be a CUDA tensor" % name)
        if t.dtype not in _DT:
            raise TypeError("%s must be float64 or float32" % name)
        if t.numel() != self.N:
            raise ValueError("%s has %d elements, operator has %d" % (name, t.numel(), self.N))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
        return t

    def workspace(self, solver: int, dtype: torch.dtype, maxit: int, device, opts=None) -> torch.Tensor:
        """Device workspace for a solver (cached per size on this operator)."""
        size = ctypes.c_size_t()
        optr = ctypes.byref(opts) if opts is not None else None
        check(_lib.load().hs_workspace_size(self._op, solver, _DT[dtype], optr, int(maxit), ctypes.byref(size)),
              "hs_workspace_size")
        key = (str(device), size.value)
        ws = self._ws.get(key)
        if ws is None:
            self._ws.clear()
            ws = torch.empty(max(size.value, 256), dtype=torch.uint8, device=device)
            self._ws[key] = ws
        return ws

    # -- operator application -----------------------------------------------
    def spmv(self, x: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """y = A x."""
        self._vec(x, "x")
        y = torch.empty_like(x) if out is None else self._vec(out, "out")
        with torch.cuda.device(x.device):
            st = torch.cuda.current_stream(x.device).cuda_stream
            check(_lib.load().hs_spmv(self._op, _DT[x.dtype], ctypes.c_void_p(x.data_ptr()),
                                      ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(st)), "hs_spmv")
        return y

    def residual(self, b: torch.Tensor, x: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """r = b - A x."""
        self._vec(b, "b")
        self._vec(x, "x")
        r = torch.empty_like(x) if out is None else self._vec(out, "out")
        with torch.cuda.device(x.device):
            st = torch.cuda.current_stream(x.device).cuda_stream
            check(_lib.load().hs_residual(self._op, _DT[x.dtype], ctypes.c_void_p(b.data_ptr()),
                                          ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(r.data_ptr()),
                                          ctypes.c_void_p(st)), "hs_residual")
        return r


def make_opts(**kw) -> _lib.hs_opts:
    o = _lib.hs_opts()
    o.struct_size = ctypes.sizeof(_lib.hs_opts)
    o.gs_mode = _lib.HS_GS_FORWARD
    o.check_every = 1
    o.restart_eps = 1e-5
    o.true_residual = 1
    o.timeout_s = 2.0
    o.inner_tol = 1e-5
    o.inner_solver = _lib.HS_SOLVER_CG
    o.inner_maxit = 10000
    o.use_graph = 1
    o.sweeps_per_pass = 1
    for k, v in kw.items():
        if k == "gs_mode" and isinstance(v, str):
            v = _GS_MODES[v]
        if k == "inner_solver" and isinstance(v, str):
            v = {"cg": _lib.HS_SOLVER_CG, "bicgstab": _lib.HS_SOLVER_BICGSTAB}[v]
        if k in ("true_residual", "use_graph", "paper_order", "inner_fixed_tol"):
            v = int(bool(v))
        if not hasattr(o, k):
            raise TypeError("unknown solver option %r" % k)
        setattr(o, k, v)
    return o


_SOLVER_FN = {
    _lib.HS_SOLVER_JACOBI: "hs_jacobi",
    _lib.HS_SOLVER_GAUSS_SEIDEL: "hs_gauss_seidel",
    _lib.HS_SOLVER_CG: "hs_cg",
    _lib.HS_SOLVER_BICGSTAB: "hs_bicgstab",
    _lib.HS_SOLVER_CG_NB: "hs_cg_nb",
}


def _solve(solver: int, A: Operator, b: torch.Tensor, x0, tol, maxit, history, inplace=False, trace=False, **kw):
    A._vec(b, "b")
    if x0 is None:
        x = torch.zeros_like(b)
    else:
        A._vec(x0, "x0")
        if x0.dtype != b.dtype:
            raise TypeError("x0 and b must have the same dtype")
        x = x0 if inplace else x0.clone()
    opts = make_opts(**kw)
    alpha = restarts_at = None
    if trace:
        alpha = np.full(int(maxit) + 1, np.nan)
        restarts_at = np.zeros(max(int(maxit), 1), dtype=np.int32)
        opts.alpha_trace = alpha.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        opts.restart_iters = restarts_at.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    res = _lib.hs_result()
    hist = np.full(int(maxit) + 1, np.nan) if history else None
    hptr = hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if hist is not None else None
    lib = _lib.load()
    fn = getattr(lib, _SOLVER_FN[solver])
    with torch.cuda.device(b.device):
        ws = A.workspace(solver, b.dtype, maxit, b.device)
        st = torch.cuda.current_stream(b.device).cuda_stream
        status = fn(A._op, _DT[b.dtype], ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                    float(tol), int(maxit), ctypes.byref(opts), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                    ctypes.c_void_p(st), ctypes.byref(res), hptr)
    if status in (_lib.HS_ERR_INVALID, _lib.HS_ERR_CUDA, _lib.HS_ERR_WORKSPACE):
        raise _lib.HsError(status, _SOLVER_FN[solver])
    if hist is not None:
        hist = hist[: res.iters + 1]
    info = SolveInfo(iters=res.iters, status=_lib.STATUS_NAMES.get(res.status, str(res.status)),
                     status_code=res.status, rel_res=res.rel_res, true_rel_res=res.true_rel_res,
                     restarts=res.restarts, history=hist, outer=res.outer, inner_iters=res.inner_iters)
    if trace:
        info.alpha_trace = alpha[: res.iters + 1]
        info.restart_iters = [int(v) for v in restarts_at[: res.restarts]]
    return x, info


def solve_mixed(A: Operator, b, x0=None, tol: float = 1e-10, maxit: int = 20, history: bool = True,
                inner_tol: float = 1e-5, inner_solver: str = "cg", inner_maxit: int = 10000, inplace=False, **kw):
    """Mixed-precision iterative refinement: FP64 residual and update, FP32 inner
    CG / BiCGStab with FP64-accumulated dots.  b, x0: float64 CUDA tensors."""
    A._vec(b, "b")
    if b.dtype != torch.float64:
        raise TypeError("solve_mixed takes float64 b and x")
    if x0 is None:
        x = torch.zeros_like(b)
    else:
        A._vec(x0, "x0")
        x = x0 if inplace else x0.clone()
    opts = make_opts(inner_tol=inner_tol, inner_solver=inner_solver, inner_maxit=inner_maxit, **kw)
    res = _lib.hs_result()
    hist = np.full(int(maxit) + 1, np.nan) if history else None
    hptr = hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if hist is not None else None
    lib = _lib.load()
    with torch.cuda.device(b.device):
        ws = A.workspace(_lib.HS_SOLVER_MIXED, torch.float64, maxit, b.device, opts)
        st = torch.cuda.current_stream(b.device).cuda_stream
        status = lib.hs_solve_mixed(A._op, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                    float(tol), int(maxit), ctypes.byref(opts), ctypes.c_void_p(ws.data_ptr()),
                                    ws.numel(), ctypes.c_void_p(st), ctypes.byref(res), hptr)
    if status in (_lib.HS_ERR_INVALID, _lib.HS_ERR_CUDA, _lib.HS_ERR_WORKSPACE):
        raise _lib.HsError(status, "hs_solve_mixed")
    if hist is not None:
        hist = hist[: res.iters + 1]
    return x, SolveInfo(iters=res.iters, status=_lib.STATUS_NAMES.get(res.status, str(res.status)),
                        status_code=res.status, rel_res=res.rel_res, true_rel_res=res.true_rel_res,
                        restarts=res.restarts, history=hist, outer=res.outer, inner_iters=res.inner_iters)


def jacobi(A: Operator, b, x0=None, tol: float = 0.0, maxit: int = 100, history: bool = False, **kw):
    """Jacobi sweeps (section 3.1); tol = 0 runs exactly maxit sweeps."""
    return _solve(_lib.HS_SOLVER_JACOBI, A, b, x0, tol, maxit, history, **kw)


def gauss_seidel(A: Operator, b, x0=None, tol: float = 0.0, maxit: int = 100, mode: str = "forward",
                 history: bool = False, **kw):
    """Exactly lexicographic Gauss-Seidel (forward / backward / symmetric)."""
    return _solve(_lib.HS_SOLVER_GAUSS_SEIDEL, A, b, x0, tol, maxit, history, gs_mode=mode, **kw)


def cg(A: Operator, b, x0=None, tol: float = 1e-10, maxit: int = 10000, history: bool = True, **kw):
    """Classical conjugate gradient with fused stencil/vector passes."""
    return _solve(_lib.HS_SOLVER_CG, A, b, x0, tol, maxit, history, **kw)


def cg_nb(A: Operator, b, x0=None, tol: float = 1e-10, maxit: int = 10000, history: bool = True, **kw):
    """CG-NB (the paper's Algorithm 1): SpMV on r, A p by recurrence, one fused
    pass and one grid reduction per iteration.  paper_order=True applies the
    printed final step x = x_l + alpha_l p_l."""
    return _solve(_lib.HS_SOLVER_CG_NB, A, b, x0, tol, maxit, history, **kw)


def bicgstab(A: Operator, b, x0=None, tol: float = 1e-10, maxit: int = 10000, history: bool = True,
             restart_eps: float = 1e-5, **kw):
    """BiCGStab with Algorithm 2's normalised shadow residual and restart;
    paper_order=True gives Algorithm 2's statement order (BiCGStab-B1);
    trace=True also returns info.alpha_trace (r_k . r' after each iteration,
    the value the restart test reads) and info.restart_iters."""
    return _solve(_lib.HS_SOLVER_BICGSTAB, A, b, x0, tol, maxit, history, restart_eps=restart_eps, **kw)


DIAG_WAITS = {"grid_barrier": 0, "gs_tile": 1, "gs27_ring": 2, "gs27_planes": 3}


def diag_wait_timeout(kind: str, timeout_s: float = 0.05) -> str:
    """Run one of the library's bounded device-side waits against a condition
    that never comes true; returns the status name ("ERR_TIMEOUT" when the
    wait gave up as designed).  The CUDA context stays usable."""
    lib = _lib.load()
    stream = torch.cuda.current_stream().cuda_stream
    st = lib.hs_diag_wait_timeout(DIAG_WAITS[kind], float(timeout_s), ctypes.c_void_p(stream))
    if st not in (_lib.HS_OK, _lib.HS_ERR_TIMEOUT):
        _lib.check(st, "hs_diag_wait_timeout")
    return _lib.STATUS_NAMES.get(st, str(st))


_ASYNC_FN = {"jacobi": ("hs_jacobi_async", _lib.HS_SOLVER_JACOBI),
             "gauss_seidel": ("hs_gauss_seidel_async", _lib.HS_SOLVER_GAUSS_SEIDEL),
             "cg": ("hs_cg_async", _lib.HS_SOLVER_CG),
             "bicgstab": ("hs_bicgstab_async", _lib.HS_SOLVER_BICGSTAB)}


class AsyncSolve:
    """A solve enqueued on the current stream with nothing on the host waiting
    (hs_jacobi_async / hs_gauss_seidel_async / hs_cg_async / hs_bicgstab_async):
    the outcome and the history land in device buffers owned by this object,
    so launch() can be captured in a CUDA graph and replayed after new values
    are copied into b and x.  b and x are used in place; the object keeps its
    own workspace.  result() copies the outcome to the host (synchronising)."""

    def __init__(self, solver: str, A: Operator, b: torch.Tensor, x: torch.Tensor, tol: float = 1e-10,
                 maxit: int = 10000, history: bool = False, **kw):
        if solver not in _ASYNC_FN:
            raise ValueError("solver must be one of %s" % sorted(_ASYNC_FN))
        A._vec(b, "b")
        A._vec(x, "x")
        if x.dtype != b.dtype or x.device != b.device:
            raise TypeError("x and b must have the same dtype and device")
        if solver == "gauss_seidel" and "mode" in kw:
            kw["gs_mode"] = kw.pop("mode")
        self.fn, code = _ASYNC_FN[solver]
        self.A, self.b, self.x = A, b, x
        self.tol, self.maxit = float(tol), int(maxit)
        self.opts = make_opts(**kw)
        size = ctypes.c_size_t()
        with torch.cuda.device(b.device):
            check(_lib.load().hs_workspace_size(A._op, code, _DT[b.dtype], ctypes.byref(self.opts), self.maxit,
                                                ctypes.byref(size)), "hs_workspace_size")
        self.ws = torch.empty(max(size.value, 256), dtype=torch.uint8, device=b.device)
        self.res = torch.zeros(ctypes.sizeof(_lib.hs_result), dtype=torch.uint8, device=b.device)
        self.hist = torch.full((self.maxit + 1,), float("nan"), dtype=torch.float64, device=b.device) if history \
            else None

    def launch(self, stream=None):
        """Enqueue the solve on `stream` (default: the current stream)."""
        lib = _lib.load()
        with torch.cuda.device(self.b.device):
            st = (stream or torch.cuda.current_stream(self.b.device)).cuda_stream
            status = getattr(lib, self.fn)(self.A._op, _DT[self.b.dtype], ctypes.c_void_p(self.b.data_ptr()),
                                           ctypes.c_void_p(self.x.data_ptr()), self.tol, self.maxit,
                                           ctypes.byref(self.opts), ctypes.c_void_p(self.ws.data_ptr()),
                                           self.ws.numel(), ctypes.c_void_p(st), ctypes.c_void_p(self.res.data_ptr()),
                                           ctypes.c_void_p(self.hist.data_ptr()) if self.hist is not None else None)
        check(status, self.fn)

    def result(self) -> SolveInfo:
        """The outcome of the last completed launch (copies it to the host)."""
        raw = self.res.cpu().numpy().tobytes()
        r = _lib.hs_result.from_buffer_copy(raw)
        hist = None
        if self.hist is not None:
            hist = self.hist[: min(r.iters, self.maxit) + 1].cpu().numpy()
        return SolveInfo(iters=r.iters, status=_lib.STATUS_NAMES.get(r.status, str(r.status)), status_code=r.status,
                         rel_res=r.rel_res, true_rel_res=r.true_rel_res, restarts=r.restarts, history=hist,
                         outer=r.outer, inner_iters=r.inner_iters)


def fp64_rate() -> float:
    """FP64 fused multiply-add rate of the current device in flop/s (the peak
    the FP64 solvers' flop rates are quoted against)."""
    v = ctypes.c_double()
    check(_lib.load().hs_diag_fp64_rate(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), ctypes.byref(v)),
          "hs_diag_fp64_rate")
    return v.value


def grad_logk(A: Operator, u: torch.Tensor, lam: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """dL/dlog k per cell from the forward solution u and the adjoint lam (float64)."""
    if A.kind != "diffusion":
        raise ValueError("grad_logk needs a diffusion operator")
    for t, n in ((u, "u"), (lam, "lam")):
        A._vec(t, n)
        if t.dtype != torch.float64:
            raise TypeError("%s must be float64" % n)
    g = torch.empty_like(u) if out is None else A._vec(out, "out")
    with torch.cuda.device(u.device):
        st = torch.cuda.current_stream(u.device).cuda_stream
        check(_lib.load().hs_diffusion_grad_logk(A._op, ctypes.c_void_p(u.data_ptr()),
                                                 ctypes.c_void_p(lam.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                                                 ctypes.c_void_p(st)), "hs_diffusion_grad_logk")
    return g


def exp_logk(logk: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """k = exp(logk) on the GPU (hs_exp_logk): the diffusion coefficient field
    from its logarithm.  logk: contiguous float64 CUDA tensor."""
    if not isinstance(logk, torch.Tensor) or not logk.is_cuda or logk.dtype != torch.float64:
        raise TypeError("logk must be a float64 CUDA tensor")
    if not logk.is_contiguous():
        raise ValueError("logk must be contiguous")
    if out is None:
        out = torch.empty_like(logk)
    elif out.shape != logk.shape or out.dtype != torch.float64 or not out.is_contiguous() or out.device != logk.device:
        raise ValueError("out must be a contiguous float64 tensor shaped like logk on its device")
    with torch.cuda.device(logk.device):
        st = torch.cuda.current_stream(logk.device).cuda_stream
        check(_lib.load().hs_exp_logk(ctypes.c_void_p(logk.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                      logk.numel(), ctypes.c_void_p(st)), "hs_exp_logk")
    return out


class DiffusionSolve(torch.autograd.Function):
    """u = A(exp(logk))^{-1} f for the variable-coefficient diffusion operator,
    differentiable in logk and f.  The backward pass solves the adjoint system
    A lam = dL/du (A is symmetric) with the same solver as the forward pass and
    returns dL/dlogk from the per-cell gradient kernel and dL/df = lam."""

    @staticmethod
    def forward(ctx, logk, f, shape, tol=1e-12, mixed=False, maxit=100000):
        k = exp_logk(logk.detach().contiguous())
        A = Operator.diffusion(shape, k)
        fd = f.detach().contiguous()
        if mixed:
            u, info = solve_mixed(A, fd, tol=tol, maxit=60, inner_maxit=maxit)
        else:
            u, info = cg(A, fd, tol=tol, maxit=maxit, history=False)
        if info.status_code < 0 or info.status_code == _lib.HS_NOT_CONVERGED:
            raise RuntimeError("forward diffusion solve failed: %s" % info.status)
        ctx.A, ctx.tol, ctx.mixed, ctx.maxit = A, tol, mixed, maxit
        ctx.save_for_backward(u)
        ctx.info = info
        return u

    @staticmethod
    def backward(ctx, grad_u):
        (u,) = ctx.saved_tensors
        A = ctx.A
        rhs = grad_u.detach().contiguous().to(torch.float64)
        if ctx.mixed:
            lam, info = solve_mixed(A, rhs, tol=ctx.tol, maxit=60, inner_maxit=ctx.maxit)
        else:
            lam, info = cg(A, rhs, tol=ctx.tol, maxit=ctx.maxit, history=False)
        if info.status_code < 0 or info.status_code == _lib.HS_NOT_CONVERGED:
            raise RuntimeError("adjoint diffusion solve failed: %s" % info.status)
        g = grad_logk(A, u, lam)
        return g, lam, None, None, None, None


def diffusion_solve(logk: torch.Tensor, f: torch.Tensor, shape, tol: float = 1e-12, mixed: bool = False,
                    maxit: int = 100000) -> torch.Tensor:
    """Differentiable solve of -div(exp(logk) grad u) = f (float64 CUDA tensors)."""
    return DiffusionSolve.apply(logk, f, tuple(shape), tol, mixed, maxit)


def batch_solve(ops, solvers, bs, xs=None, tol: float = 1e-8, maxit: int = 20000, stream=None, **kw):
    """Solve many independent systems with one persistent kernel (a Batch built
    for these operators and solvers, then Batch.solve); returns (xs, infos)."""
    return Batch(ops, solvers).solve(bs, xs, tol=tol, maxit=maxit, stream=stream, **kw)


class Batch:
    """Many independent systems solved by one persistent kernel (CUDA graph).

    ops: list of Operators; solvers: list of "cg" / "bicgstab" (one per system),
    or "mixed" for every system: FP64 iterative refinement per system with an
    FP32 inner CG (symmetric operators) or BiCGStab (upwind operator); then
    maxit bounds the refinement steps and inner_tol / inner_maxit the inner
    solves.
    """

    def __init__(self, ops, solvers, autotune: bool = False):
        lib = _lib.load()
        if len(ops) != len(solvers) or not ops:
            raise ValueError("need one solver per operator")
        self.ops = list(ops)
        self.n = len(ops)
        code = {"cg": _lib.HS_SOLVER_CG, "bicgstab": _lib.HS_SOLVER_BICGSTAB, "mixed": _lib.HS_SOLVER_MIXED}
        self.mixed = solvers[0] == "mixed"
        arr_ops = (ctypes.c_void_p * self.n)(*[o._op.value for o in self.ops])
        arr_sol = (ctypes.c_int * self.n)(*[code[s] for s in solvers])
        self._b = ctypes.c_void_p()
        check(lib.hs_batch_create(self.n, arr_ops, arr_sol, ctypes.byref(self._b)), "hs_batch_create")
        self._ws = None
        self.tile_planes = None
        if autotune:
            from .autotune import batch_tile_planes
            self.tile_planes = batch_tile_planes(self.ops, list(solvers))
            arr = (ctypes.c_int * self.n)(*self.tile_planes)
            check(lib.hs_batch_set_tile_planes(self._b, arr), "hs_batch_set_tile_planes")

    def __del__(self):
        try:
            if self._b is not None and self._b.value:
                _lib.load().hs_batch_destroy(self._b)
                self._b = None
        except Exception:
            pass

    def workspace(self, device) -> torch.Tensor:
        size = ctypes.c_size_t()
        with torch.cuda.device(device):
            check(_lib.load().hs_batch_workspace_size(self._b, ctypes.byref(size)), "hs_batch_workspace_size")
        if self._ws is None or self._ws.numel() < size.value or self._ws.device != torch.device(device):
            self._ws = torch.empty(max(size.value, 256), dtype=torch.uint8, device=device)
        return self._ws

    @property
    def teams(self):
        t = (ctypes.c_int * self.n)()
        check(_lib.load().hs_batch_team_sizes(self._b, t), "hs_batch_team_sizes")
        return list(t)

    @property
    def graph_used(self) -> bool:
        return bool(_lib.load().hs_batch_graph_used(self._b))

    def solve(self, bs, xs=None, tol: float = 1e-8, maxit: int = 20000, stream=None, **kw):
        """Solve A_s x_s = b_s for every system; returns (xs, infos)."""
        if len(bs) != self.n:
            raise ValueError("need one right-hand side per system")
        for A, b in zip(self.ops, bs):
            A._vec(b, "b")
            if b.dtype != torch.float64:
                raise TypeError("batched solves take float64 vectors")
        xs = [torch.zeros_like(b) for b in bs] if xs is None else xs
        for A, x in zip(self.ops, xs):
            A._vec(x, "x")
        dev = bs[0].device
        opts = make_opts(**kw)
        res = (_lib.hs_result * self.n)()
        pb = (ctypes.c_void_p * self.n)(*[b.data_ptr() for b in bs])
        px = (ctypes.c_void_p * self.n)(*[x.data_ptr() for x in xs])
        with torch.cuda.device(dev):
            ws = self.workspace(dev)
            st = (stream or torch.cuda.current_stream(dev)).cuda_stream
            status = _lib.load().hs_batch_solve(self._b, pb, px, float(tol), int(maxit), ctypes.byref(opts),
                                                ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.c_void_p(st), res)
        if status in (_lib.HS_ERR_INVALID, _lib.HS_ERR_CUDA, _lib.HS_ERR_WORKSPACE):
            raise _lib.HsError(status, "hs_batch_solve")
        infos = [SolveInfo(iters=r.iters, status=_lib.STATUS_NAMES.get(r.status, str(r.status)), status_code=r.status,
                           rel_res=r.rel_res, true_rel_res=r.true_rel_res, restarts=r.restarts, outer=r.outer,
                           inner_iters=r.inner_iters) for r in res]
        return xs, infos
