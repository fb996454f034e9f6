"""ctypes declarations of the libhsolve C ABI (include/hsolve.h).

Argument marshalling only: every numerical step runs in the CUDA library.
Loading fails loudly when the library has not been built -- there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

HS_OK = 0
HS_NOT_CONVERGED = 1
HS_ERR_INVALID = -1
HS_ERR_CUDA = -2
HS_ERR_BREAKDOWN = -3
HS_ERR_NONFINITE = -4
HS_ERR_TIMEOUT = -5
HS_ERR_WORKSPACE = -6
HS_ERR_BOUNDS = -7

STATUS_NAMES = {0: "OK", 1: "NOT_CONVERGED", -1: "ERR_INVALID", -2: "ERR_CUDA", -3: "ERR_BREAKDOWN",
                -4: "ERR_NONFINITE", -5: "ERR_TIMEOUT", -6: "ERR_WORKSPACE",
                -7: "ERR_BOUNDS"}

HS_F64, HS_F32 = 0, 1
HS_SOLVER_JACOBI, HS_SOLVER_GAUSS_SEIDEL, HS_SOLVER_CG, HS_SOLVER_BICGSTAB, HS_SOLVER_MIXED, HS_SOLVER_CG_NB = 0, 1, 2, 3, 4, 5
HS_GS_FORWARD, HS_GS_BACKWARD, HS_GS_SYMMETRIC = 0, 1, 2
HS_STATIC_SCRATCH_BYTES = 16 << 20   # include/hsolve.h


class hs_opts(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_size_t),
                ("gs_mode", ctypes.c_int),
                ("check_every", ctypes.c_int),
                ("restart_eps", ctypes.c_double),
                ("true_residual", ctypes.c_int),
                ("timeout_s", ctypes.c_double),
                ("inner_tol", ctypes.c_double),
                ("inner_solver", ctypes.c_int),
                ("inner_maxit", ctypes.c_int),
                ("use_graph", ctypes.c_int),
                ("tile_rows", ctypes.c_int),
                ("tile_planes", ctypes.c_int),
                ("max_blocks", ctypes.c_int),
                ("paper_order", ctypes.c_int),
                ("sweeps_per_pass", ctypes.c_int),
                ("alpha_trace", ctypes.POINTER(ctypes.c_double)),
                ("restart_iters", ctypes.POINTER(ctypes.c_int)),
                ("staging", ctypes.c_int),
                ("inner_fixed_tol", ctypes.c_int),
                ("gs_schedule", ctypes.c_int)]


class hs_result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int),
                ("status", ctypes.c_int),
                ("rel_res", ctypes.c_double),
                ("true_rel_res", ctypes.c_double),
                ("restarts", ctypes.c_int),
                ("outer", ctypes.c_int),
                ("inner_iters", ctypes.c_longlong)]


# Every symbol declared in include/hsolve.h, with (restype, argtypes).
_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double
_sz = ctypes.c_size_t
SIGNATURES = {
    "hs_grid_create": (_i, [_i, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_vp)]),
    "hs_grid_destroy": (None, [_vp]),
    "hs_op_laplacian": (_i, [_vp, ctypes.POINTER(_vp)]),
    "hs_op_hpcg": (_i, [_vp, _i, ctypes.POINTER(_vp)]),
    "hs_op_convdiff_upwind": (_i, [_vp, ctypes.POINTER(_d), ctypes.POINTER(_vp)]),
    "hs_op_diffusion": (_i, [_vp, _i, _vp, ctypes.POINTER(_vp)]),
    "hs_op_destroy": (None, [_vp]),
    "hs_op_size": (ctypes.c_int64, [_vp]),
    "hs_spmv": (_i, [_vp, _i, _vp, _vp, _vp]),
    "hs_residual": (_i, [_vp, _i, _vp, _vp, _vp, _vp]),
    "hs_workspace_size": (_i, [_vp, _i, _i, ctypes.POINTER(hs_opts), _i, ctypes.POINTER(_sz)]),
    "hs_jacobi": (_i, [_vp, _i, _vp, _vp, _d, _i, ctypes.POINTER(hs_opts), _vp, _sz, _vp,
                       ctypes.POINTER(hs_result), ctypes.POINTER(_d)]),
    "hs_gauss_seidel": (_i, [_vp, _i, _vp, _vp, _d, _i, ctypes.POINTER(hs_opts), _vp, _sz, _vp,
                             ctypes.POINTER(hs_result), ctypes.POINTER(_d)]),
    "hs_cg": (_i, [_vp, _i, _vp, _vp, _d, _i, ctypes.POINTER(hs_opts), _vp, _sz, _vp,
                   ctypes.POINTER(hs_result), ctypes.POINTER(_d)]),
    "hs_cg_nb": (_i, [_vp, _i, _vp, _vp, _d, _i, ctypes.POINTER(hs_opts), _vp, _sz, _vp,
                   ctypes.POINTER(hs_result), ctypes.POINTER(_d)]),
    "hs_bicgstab": (_i, [_vp, _i, _vp, _vp, _d, _i, ctypes.POINTER(hs_opts), _vp, _sz, _vp,
                         ctypes.POINTER(hs_result), ctypes.POINTER(_d)]),
    "hs_jacobi_async": (_i, [_vp, _i, _vp, _vp, _d, _i, ctypes.POINTER(hs_opts), _vp, _sz, _vp, _vp, _vp]),
    "hs_gauss_seidel_async": (_i, [_vp, _i, _vp, _vp, _d, _i, ctypes.POINTER(hs_opts), _vp, _sz, _vp, _vp, _vp]),
    "hs_cg_async": (_i, [_vp, _i, _vp, _vp, _d, _i, ctypes.POINTER(hs_opts), _vp, _sz, _vp, _vp, _vp]),
    "hs_bicgstab_async": (_i, [_vp, _i, _vp, _vp, _d, _i, ctypes.POINTER(hs_opts), _vp, _sz, _vp, _vp, _vp]),
    "hs_solve_mixed": (_i, [_vp, _vp, _vp, _d, _i, ctypes.POINTER(hs_opts), _vp, _sz, _vp,
                            ctypes.POINTER(hs_result), ctypes.POINTER(_d)]),
    "hs_diffusion_grad_logk": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "hs_exp_logk": (_i, [_vp, _vp, ctypes.c_int64, _vp]),
    "hs_cg_static": (_i, [_vp, _i, _vp, _vp, _d, _i, ctypes.POINTER(hs_opts), _vp,
                          ctypes.POINTER(hs_result), ctypes.POINTER(_d)]),
    "hs_batch_create": (_i, [_i, ctypes.POINTER(_vp), ctypes.POINTER(_i), ctypes.POINTER(_vp)]),
    "hs_batch_destroy": (None, [_vp]),
    "hs_batch_workspace_size": (_i, [_vp, ctypes.POINTER(_sz)]),
    "hs_batch_solve": (_i, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _d, _i, ctypes.POINTER(hs_opts), _vp, _sz,
                            _vp, ctypes.POINTER(hs_result)]),
    "hs_batch_set_tile_planes": (_i, [_vp, ctypes.POINTER(_i)]),
    "hs_batch_graph_used": (_i, [_vp]),
    "hs_batch_grid": (_i, [_vp]),
    "hs_batch_team_sizes": (_i, [_vp, ctypes.POINTER(_i)]),
    "hs_diag_wait_timeout": (_i, [_i, ctypes.c_double, _vp]),
    "hs_diag_fp64_rate": (_i, [_vp, ctypes.POINTER(_d)]),
    "hs_last_error": (ctypes.c_char_p, []),
    "hs_last_staging": (_i, []),
    "hs_version": (ctypes.c_char_p, []),
}

_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libhsolve.so (building it first if allowed); raise if unavailable."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError("libhsolve.so is not built (%s); run paper_2305_05988_gb300._build.build()" % path)
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


class HsError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = load().hs_last_error().decode(errors="replace")
        super().__init__("%s failed: %s (%s)" % (where, STATUS_NAMES.get(status, status), msg))
        self.status = status


def check(status: int, where: str):
    if status < 0:
        raise HsError(status, where)
    return status
