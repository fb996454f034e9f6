"""The C-ABI library builds, loads and exports every declared symbol; host-only
entry points validate their arguments.  No GPU needed (no kernel is launched)."""
import ctypes
import os
import re

import pytest

from paper_2305_05988_gb300 import _build, _lib, solvers

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(hs_[a-z0-9_]+)\s*\(", text))
    return names


def _gpu_visible():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


# These tests hand fake device addresses to entry points that must reject the
# call before touching the GPU.  They run only where no GPU is visible, so a
# regression in the validation order can never send a bogus pointer to a kernel.
no_gpu_only = pytest.mark.skipif(_gpu_visible(), reason="fake-pointer validation tests run on CPU-only hosts")


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported_and_bound(lib):
    decl = declared_symbols()
    assert len(decl) >= 16
    for name in sorted(decl):
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, "binding misses " + name


def test_version_and_error_strings(lib):
    assert b"sm_103a" in lib.hs_version()
    assert isinstance(lib.hs_last_error(), bytes)


def test_grid_validation(lib):
    g = ctypes.c_void_p()
    n = (ctypes.c_int64 * 3)(4, 0, 1)
    assert lib.hs_grid_create(2, n, ctypes.byref(g)) == _lib.HS_ERR_INVALID
    assert b"n[1]" in lib.hs_last_error()
    assert lib.hs_grid_create(4, (ctypes.c_int64 * 3)(1, 1, 1), ctypes.byref(g)) == _lib.HS_ERR_INVALID
    big = (ctypes.c_int64 * 3)(2048, 2048, 1024)
    assert lib.hs_grid_create(3, big, ctypes.byref(g)) == _lib.HS_ERR_INVALID
    assert lib.hs_grid_create(3, (ctypes.c_int64 * 3)(5, 6, 7), ctypes.byref(g)) == _lib.HS_OK
    op = ctypes.c_void_p()
    beta_bad = (ctypes.c_double * 3)(1.0, -0.5, 0.0)
    assert lib.hs_op_convdiff_upwind(g, beta_bad, ctypes.byref(op)) == _lib.HS_ERR_INVALID
    assert lib.hs_op_diffusion(g, _lib.HS_F64, None, ctypes.byref(op)) == _lib.HS_ERR_INVALID
    assert lib.hs_op_laplacian(g, ctypes.byref(op)) == _lib.HS_OK
    assert lib.hs_op_size(op) == 210
    lib.hs_grid_destroy(g)
    # workspace sizes grow with the number of solver vectors
    sizes = {}
    for s in (0, 1, 2, 3):
        b = ctypes.c_size_t()
        assert lib.hs_workspace_size(op, s, _lib.HS_F64, None, 100, ctypes.byref(b)) == _lib.HS_OK
        sizes[s] = b.value
    assert sizes[3] > sizes[2] > sizes[0] > 0
    b32 = ctypes.c_size_t()
    lib.hs_workspace_size(op, 2, _lib.HS_F32, None, 100, ctypes.byref(b32))
    assert b32.value < sizes[2]
    assert lib.hs_workspace_size(op, 7, _lib.HS_F64, None, 100, ctypes.byref(b32)) == _lib.HS_ERR_INVALID
    lib.hs_op_destroy(op)


@no_gpu_only
def test_solver_rejects_bad_arguments_without_touching_the_gpu(lib):
    g = ctypes.c_void_p()
    lib.hs_grid_create(2, (ctypes.c_int64 * 3)(8, 8, 1), ctypes.byref(g))
    op = ctypes.c_void_p()
    lib.hs_op_laplacian(g, ctypes.byref(op))
    lib.hs_grid_destroy(g)
    res = _lib.hs_result()
    # null b / x
    st = lib.hs_cg(op, 0, None, None, 1e-8, 10, None, None, 0, None, ctypes.byref(res), None)
    assert st == _lib.HS_ERR_INVALID and res.status == _lib.HS_ERR_INVALID
    # misaligned vectors
    st = lib.hs_cg(op, 0, ctypes.c_void_p(0x1008), ctypes.c_void_p(0x2000), 1e-8, 10, None, None, 0, None,
                   ctypes.byref(res), None)
    assert st == _lib.HS_ERR_INVALID
    # negative tolerance, negative maxit
    st = lib.hs_jacobi(op, 0, ctypes.c_void_p(0x1000), ctypes.c_void_p(0x2000), -1.0, 10, None, None, 0, None,
                       ctypes.byref(res), None)
    assert st == _lib.HS_ERR_INVALID
    st = lib.hs_jacobi(op, 0, ctypes.c_void_p(0x1000), ctypes.c_void_p(0x2000), 0.0, -3, None, None, 0, None,
                       ctypes.byref(res), None)
    assert st == _lib.HS_ERR_INVALID
    # missing / small / misaligned workspace
    st = lib.hs_jacobi(op, 0, ctypes.c_void_p(0x1000), ctypes.c_void_p(0x2000), 0.0, 3, None, None, 0, None,
                       ctypes.byref(res), None)
    assert st == _lib.HS_ERR_WORKSPACE
    st = lib.hs_jacobi(op, 0, ctypes.c_void_p(0x1000), ctypes.c_void_p(0x2000), 0.0, 3, None,
                       ctypes.c_void_p(0x10000), 64, None, ctypes.byref(res), None)
    assert st == _lib.HS_ERR_WORKSPACE and b"too small" in lib.hs_last_error()
    st = lib.hs_jacobi(op, 0, ctypes.c_void_p(0x1000), ctypes.c_void_p(0x2000), 0.0, 3, None,
                       ctypes.c_void_p(0x10010), 1 << 30, None, ctypes.byref(res), None)
    assert st == _lib.HS_ERR_WORKSPACE and b"aligned" in lib.hs_last_error()
    # bad options
    o = _lib.hs_opts()
    o.struct_size = 0
    st = lib.hs_bicgstab(op, 0, ctypes.c_void_p(0x1000), ctypes.c_void_p(0x2000), 1e-8, 3, ctypes.byref(o),
                         ctypes.c_void_p(0x100000), 1 << 30, None, ctypes.byref(res), None)
    assert st == _lib.HS_ERR_INVALID
    # option values outside their ranges
    for field, bad in (("gs_schedule", 4), ("gs_schedule", -1), ("staging", 2), ("gs_mode", 5)):
        o = solvers.make_opts()
        setattr(o, field, bad)
        st = lib.hs_gauss_seidel(op, 0, ctypes.c_void_p(0x1000), ctypes.c_void_p(0x2000), 0.0, 3, ctypes.byref(o),
                                 ctypes.c_void_p(0x100000), 1 << 30, None, ctypes.byref(res), None)
        assert st == _lib.HS_ERR_INVALID, (field, bad)
    lib.hs_op_destroy(op)


@no_gpu_only
def test_cg_rejects_nonsymmetric_operator(lib):
    g = ctypes.c_void_p()
    lib.hs_grid_create(2, (ctypes.c_int64 * 3)(8, 8, 1), ctypes.byref(g))
    op = ctypes.c_void_p()
    lib.hs_op_convdiff_upwind(g, (ctypes.c_double * 3)(3.0, 1.0, 0.0), ctypes.byref(op))
    lib.hs_grid_destroy(g)
    res = _lib.hs_result()
    st = lib.hs_cg(op, 0, ctypes.c_void_p(0x1000), ctypes.c_void_p(0x2000), 1e-8, 3, None,
                   ctypes.c_void_p(0x100000), 1 << 30, None, ctypes.byref(res), None)
    assert st == _lib.HS_ERR_INVALID and b"symmetric" in lib.hs_last_error()
    lib.hs_op_destroy(op)


def test_hpcg_operator_validation_and_workspace(lib):
    g2, g3 = ctypes.c_void_p(), ctypes.c_void_p()
    lib.hs_grid_create(2, (ctypes.c_int64 * 3)(8, 6, 1), ctypes.byref(g2))
    lib.hs_grid_create(3, (ctypes.c_int64 * 3)(8, 6, 5), ctypes.byref(g3))
    op = ctypes.c_void_p()
    assert lib.hs_op_hpcg(g3, 5, ctypes.byref(op)) == _lib.HS_ERR_INVALID
    assert lib.hs_op_hpcg(g2, 27, ctypes.byref(op)) == _lib.HS_ERR_INVALID
    assert b"3-D" in lib.hs_last_error()
    op7, op27 = ctypes.c_void_p(), ctypes.c_void_p()
    assert lib.hs_op_hpcg(g2, 7, ctypes.byref(op7)) == _lib.HS_OK
    assert lib.hs_op_hpcg(g3, 27, ctypes.byref(op27)) == _lib.HS_OK
    assert lib.hs_op_size(op27) == 240
    lib.hs_grid_destroy(g2)
    lib.hs_grid_destroy(g3)
    # CG-NB keeps r, w, q in two copies plus p: more than CG, less than BiCGStab
    sz = {}
    for s in (_lib.HS_SOLVER_CG, _lib.HS_SOLVER_CG_NB, _lib.HS_SOLVER_BICGSTAB):
        b = ctypes.c_size_t()
        assert lib.hs_workspace_size(op27, s, _lib.HS_F64, None, 50, ctypes.byref(b)) == _lib.HS_OK
        sz[s] = b.value
    assert sz[_lib.HS_SOLVER_CG] < sz[_lib.HS_SOLVER_CG_NB] < sz[_lib.HS_SOLVER_BICGSTAB]
    lib.hs_op_destroy(op7)
    lib.hs_op_destroy(op27)


@no_gpu_only
def test_cg_nb_and_batch_reject_bad_operators(lib):
    g = ctypes.c_void_p()
    lib.hs_grid_create(3, (ctypes.c_int64 * 3)(8, 8, 8), ctypes.byref(g))
    up, box = ctypes.c_void_p(), ctypes.c_void_p()
    lib.hs_op_convdiff_upwind(g, (ctypes.c_double * 3)(3.0, 1.0, 0.5), ctypes.byref(up))
    lib.hs_op_hpcg(g, 27, ctypes.byref(box))
    lib.hs_grid_destroy(g)
    res = _lib.hs_result()
    st = lib.hs_cg_nb(up, 0, ctypes.c_void_p(0x1000), ctypes.c_void_p(0x2000), 1e-8, 3, None,
                      ctypes.c_void_p(0x100000), 1 << 30, None, ctypes.byref(res), None)
    assert st == _lib.HS_ERR_INVALID and b"symmetric" in lib.hs_last_error()
    batch = ctypes.c_void_p()
    ops = (ctypes.c_void_p * 1)(box.value)
    sol = (ctypes.c_int * 1)(_lib.HS_SOLVER_CG)
    assert lib.hs_batch_create(1, ops, sol, ctypes.byref(batch)) == _lib.HS_ERR_INVALID
    assert b"7-point" in lib.hs_last_error()
    lib.hs_op_destroy(up)
    lib.hs_op_destroy(box)


def test_diag_wait_validation(lib):
    # rejected before anything reaches the GPU
    assert lib.hs_diag_wait_timeout(4, 0.1, None) == _lib.HS_ERR_INVALID
    assert lib.hs_diag_wait_timeout(-1, 0.1, None) == _lib.HS_ERR_INVALID
    assert lib.hs_diag_wait_timeout(0, 0.0, None) == _lib.HS_ERR_INVALID
    assert lib.hs_diag_wait_timeout(1, 10.5, None) == _lib.HS_ERR_INVALID
    assert lib.hs_diag_wait_timeout(2, float("nan"), None) == _lib.HS_ERR_INVALID


def test_exp_logk_validation(lib):
    # rejected (or, for n = 0, finished) before anything reaches the GPU
    vp = ctypes.c_void_p
    assert lib.hs_exp_logk(vp(4096), vp(8192), -1, None) == _lib.HS_ERR_INVALID
    assert lib.hs_exp_logk(None, vp(8192), 10, None) == _lib.HS_ERR_INVALID
    assert lib.hs_exp_logk(vp(4096), None, 10, None) == _lib.HS_ERR_INVALID
    assert lib.hs_exp_logk(None, None, 0, None) == _lib.HS_OK
    # partial overlap (k starts 8 elements into logk's 10)
    assert lib.hs_exp_logk(vp(4096), vp(4096 + 64), 10, None) == _lib.HS_ERR_INVALID
    assert lib.hs_exp_logk(vp(4096 + 64), vp(4096), 10, None) == _lib.HS_ERR_INVALID
    assert b"overlap" in lib.hs_last_error()


def test_gauss_seidel_workspace_sizes(lib):
    # GS keeps b / a_ii (one vector) plus its schedule: tile-plane tables,
    # per-tile sweep counts and a claim counter (7-point), or per-block
    # progress words (27-point); never less than the vector, never a
    # Krylov solver's several vectors
    g = ctypes.c_void_p()
    lib.hs_grid_create(3, (ctypes.c_int64 * 3)(64, 48, 40), ctypes.byref(g))
    lap, box = ctypes.c_void_p(), ctypes.c_void_p()
    assert lib.hs_op_laplacian(g, ctypes.byref(lap)) == _lib.HS_OK
    assert lib.hs_op_hpcg(g, 27, ctypes.byref(box)) == _lib.HS_OK
    lib.hs_grid_destroy(g)
    N = 64 * 48 * 40
    for op in (lap, box):
        gs, cg = ctypes.c_size_t(), ctypes.c_size_t()
        assert lib.hs_workspace_size(op, _lib.HS_SOLVER_GAUSS_SEIDEL, _lib.HS_F64, None, 10,
                                     ctypes.byref(gs)) == _lib.HS_OK
        assert lib.hs_workspace_size(op, _lib.HS_SOLVER_CG, _lib.HS_F64, None, 10, ctypes.byref(cg)) == _lib.HS_OK
        assert 8 * N < gs.value < cg.value
        gs32 = ctypes.c_size_t()
        lib.hs_workspace_size(op, _lib.HS_SOLVER_GAUSS_SEIDEL, _lib.HS_F32, None, 10, ctypes.byref(gs32))
        assert 4 * N < gs32.value < gs.value
        # the residual history grows with maxit
        big = ctypes.c_size_t()
        lib.hs_workspace_size(op, _lib.HS_SOLVER_GAUSS_SEIDEL, _lib.HS_F64, None, 100000, ctypes.byref(big))
        assert big.value > gs.value
    lib.hs_op_destroy(lap)
    lib.hs_op_destroy(box)


def test_struct_layouts_match_the_header(tmp_path):
    # the binding's ctypes structures against the C compiler's layout of the
    # header's hs_opts and hs_result (size and every field offset)
    fields = {"hs_opts": _lib.hs_opts, "hs_result": _lib.hs_result}
    src = ['#include <stddef.h>', '#include <stdio.h>', '#include "hsolve.h"', "int main(void) {"]
    for sname, cls in fields.items():
        src.append('printf("%s size %%zu\\n", sizeof(%s));' % (sname, sname))
        for fname, _ in cls._fields_:
            src.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (sname, fname, sname, fname))
    src.append("return 0; }")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(line.split()[:2]): int(line.split()[2]) for line in out if line.strip()}
    for sname, cls in fields.items():
        assert got[(sname, "size")] == ctypes.sizeof(cls), sname
        for fname, _ in cls._fields_:
            assert got[(sname, fname)] == getattr(cls, fname).offset, (sname, fname)
