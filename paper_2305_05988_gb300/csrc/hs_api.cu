// hs_api.cu -- the extern "C" surface of libhsolve: handles, argument
// validation, workspace sizing and error reporting.  The numerical work is
// in hs_kernels.cu (SpMV, Jacobi, CG, BiCGStab) and hs_gs.cu (Gauss-Seidel).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "hs_internal.h"

namespace hs {

static thread_local char g_err[512] = "no error";
static thread_local int g_last_staging = 0;

void set_last_staging(int v) { g_last_staging = v; }

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

hs_status cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
  return HS_ERR_CUDA;
}

size_t common_bytes(int maxit) {
  Carve c{nullptr, 0, (size_t)-1, true};
  carve_common(c, maxit);
  return c.off;
}

Common carve_common(Carve& c, int maxit) {
  Common cm;
  cm.ctrl = c.take<Ctrl>(1);
  // ctrl slot is 512 bytes so that later fields never move
  if (sizeof(Ctrl) < 512) c.take<char>(512 - ((sizeof(Ctrl) + 255) & ~(size_t)255));
  cm.partials = c.take<double>((size_t)MAX_BLOCKS * MAX_SCAL);
  cm.hist = c.take<double>((size_t)maxit + 2);
  return cm;
}

size_t gs_ws_vectors(const hs_op* A, hs_dtype dt);  // hs_gs.cu
size_t mixed_ws_bytes(const hs_op* A, const hs_opts& o, int max_outer);  // hs_kernels.cu
hs_status run_mixed(const SolveArgs& sa, hs_result* res, double* hist);   // hs_kernels.cu

size_t ws_bytes_for(const hs_op* A, hs_solver s, hs_dtype dt, int maxit) {
  size_t N = (size_t)(A->n[0] * A->n[1] * A->n[2]);
  size_t es = dt == HS_F64 ? 8 : 4;
  size_t vec = (N * es + 255) & ~(size_t)255;
  size_t nvec = 0;
  switch (s) {
    case HS_SOLVER_JACOBI: nvec = 2; break;
    case HS_SOLVER_CG: nvec = 4; break;
    case HS_SOLVER_BICGSTAB: nvec = 8; break;
    case HS_SOLVER_GAUSS_SEIDEL: return common_bytes(maxit) + gs_ws_vectors(A, dt) + vark_coef_bytes(A, dt);
    case HS_SOLVER_MIXED: return 0;  // sized by mixed_ws_bytes with the options
    case HS_SOLVER_CG_NB: nvec = 7; break;  // r, w, q ping-pong pairs and p
  }
  size_t extra = 0;
  if (s == HS_SOLVER_BICGSTAB) extra = (bicgstab_trace_len(maxit) * sizeof(double) + 255) & ~(size_t)255;
  return common_bytes(maxit) + nvec * vec + vark_coef_bytes(A, dt) + extra;
}

static hs_opts default_opts() {
  hs_opts o;
  memset(&o, 0, sizeof(o));
  o.struct_size = sizeof(hs_opts);
  o.gs_mode = HS_GS_FORWARD;
  o.check_every = 1;
  o.restart_eps = 1e-5;
  o.true_residual = 1;
  o.timeout_s = 2.0;
  o.inner_tol = 1e-5;
  o.inner_solver = HS_SOLVER_CG;
  o.inner_maxit = 10000;
  o.use_graph = 1;
  o.sweeps_per_pass = 1;
  return o;
}

bool merge_opts(const hs_opts* in, hs_opts* out) {
  *out = default_opts();
  if (!in) return true;
  if (in->struct_size < sizeof(size_t) || in->struct_size > 4096) {
    set_error("hs_opts.struct_size must be set to sizeof(hs_opts)");
    return false;
  }
  size_t n = in->struct_size < sizeof(hs_opts) ? in->struct_size : sizeof(hs_opts);
  memcpy(out, in, n);
  out->struct_size = sizeof(hs_opts);
  if (out->gs_mode < 0 || out->gs_mode > 2) {
    set_error("hs_opts.gs_mode out of range");
    return false;
  }
  if (out->check_every < 1) out->check_every = 1;
  if (!(out->restart_eps >= 0.0) || !isfinite(out->restart_eps)) {
    set_error("hs_opts.restart_eps must be finite and >= 0");
    return false;
  }
  if (!(out->timeout_s > 0.0) || out->timeout_s > 3600.0) out->timeout_s = 2.0;
  if (!(out->inner_tol >= 0.0) || !isfinite(out->inner_tol)) {
    set_error("hs_opts.inner_tol must be finite and >= 0");
    return false;
  }
  if (out->inner_solver != HS_SOLVER_CG && out->inner_solver != HS_SOLVER_BICGSTAB) {
    set_error("hs_opts.inner_solver must be HS_SOLVER_CG or HS_SOLVER_BICGSTAB");
    return false;
  }
  if (out->inner_maxit < 1 || out->inner_maxit > 100000000) out->inner_maxit = 10000;
  if (out->tile_planes < 0) out->tile_planes = 0;
  if (out->max_blocks < 0) out->max_blocks = 0;
  out->paper_order = out->paper_order ? 1 : 0;
  out->inner_fixed_tol = out->inner_fixed_tol ? 1 : 0;
  if (out->sweeps_per_pass < 1) out->sweeps_per_pass = 1;
  if (out->staging < 0 || out->staging > 1) {
    set_error("hs_opts.staging must be 0 (register prefetch) or 1 (TMA)");
    return false;
  }
  if (out->sweeps_per_pass > 4) out->sweeps_per_pass = 4;
  if (out->gs_schedule < 0 || out->gs_schedule > 3) {
    set_error("hs_opts.gs_schedule must be 0 (automatic), 1 (tiles), 2 (pencils) or 3 (one cluster)");
    return false;
  }
  return true;
}

static bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }


static size_t ws_need(const hs_op* A, hs_solver s, hs_dtype dt, const hs_opts& o, int maxit) {
  if (s == HS_SOLVER_MIXED) return mixed_ws_bytes(A, o, maxit);
  return ws_bytes_for(A, s, dt, maxit);
}

static hs_status check_solve(const hs_op* A, hs_dtype dt, const void* b, const void* x, double tol, int maxit,
                             const void* ws, size_t ws_bytes, hs_solver s, const hs_opts& o) {
  if (!A) { set_error("operator is NULL"); return HS_ERR_INVALID; }
  if (dt != HS_F64 && dt != HS_F32) { set_error("dtype must be HS_F64 or HS_F32"); return HS_ERR_INVALID; }
  if (!b || !x) { set_error("b and x must be device pointers"); return HS_ERR_INVALID; }
  if (!aligned(b, 16) || !aligned(x, 16)) { set_error("b and x must be 16-byte aligned"); return HS_ERR_INVALID; }
  if (b == x) { set_error("b and x must not alias"); return HS_ERR_INVALID; }
  if (!(tol >= 0.0) || !isfinite(tol)) { set_error("tol must be finite and >= 0"); return HS_ERR_INVALID; }
  if (maxit < 0 || maxit > 100000000) { set_error("maxit out of range"); return HS_ERR_INVALID; }
  if (!ws) { set_error("workspace is NULL"); return HS_ERR_WORKSPACE; }
  if (!aligned(ws, 256)) { set_error("workspace must be 256-byte aligned"); return HS_ERR_WORKSPACE; }
  size_t need = ws_need(A, s, dt, o, maxit);
  if (ws_bytes < need) {
    set_error("workspace too small: %zu bytes given, %zu needed", ws_bytes, need);
    return HS_ERR_WORKSPACE;
  }
  return HS_OK;
}

static void fill_res(hs_result* res) {
  if (!res) return;
  memset(res, 0, sizeof(*res));
  res->status = HS_ERR_INVALID;
  res->rel_res = -1.0;
  res->true_rel_res = -1.0;
}

typedef hs_status (*runner_t)(const SolveArgs&, hs_result*, double*);

static hs_status solve_common(runner_t run, hs_solver which, const hs_op* A, hs_dtype dt, const void* b, void* x,
                              double tol, int maxit, const hs_opts* opts, void* ws, size_t ws_bytes, void* stream,
                              hs_result* res, double* hist) {
  static const char* const names[] = {"hs_jacobi", "hs_gauss_seidel", "hs_cg", "hs_bicgstab", "hs_solve_mixed",
                                      "hs_cg_nb"};
  NvtxRange range(which >= 0 && which <= 5 ? names[which] : "hs_solve");
  hs_result local;
  hs_result* r = res ? res : &local;
  fill_res(r);
  hs_opts o;
  if (!merge_opts(opts, &o)) return HS_ERR_INVALID;
  hs_status s = check_solve(A, dt, b, x, tol, maxit, ws, ws_bytes, which, o);
  if (s != HS_OK) return s;
  SolveArgs a;
  a.A = A;
  a.dtype = dt;
  a.b = b;
  a.x = x;
  a.tol = tol;
  a.maxit = maxit;
  a.o = o;
  a.ws = (char*)ws;
  a.ws_bytes = ws_bytes;
  a.stream = (cudaStream_t)stream;
  cudaError_t e = cudaGetLastError();  // clear stale errors from unrelated work
  (void)e;
  s = run(a, r, hist);
  if (s == HS_ERR_CUDA || s == HS_ERR_INVALID || s == HS_ERR_WORKSPACE) r->status = s;
  return s;
}

// The asynchronous form: validated like the synchronous calls (errors are
// returned at once), then everything is enqueued on the stream and the result
// and the history are written by a kernel into device memory.
static hs_status solve_async(runner_t run, hs_solver which, const hs_op* A, hs_dtype dt, const void* b, void* x,
                             double tol, int maxit, const hs_opts* opts, void* ws, size_t ws_bytes, void* stream,
                             hs_result* res_dev, double* hist_dev) {
  static const char* const names[] = {"hs_jacobi_async", "hs_gauss_seidel_async", "hs_cg_async",
                                      "hs_bicgstab_async", "hs_solve_mixed", "hs_cg_nb_async"};
  NvtxRange range(which >= 0 && which <= 5 ? names[which] : "hs_solve_async");
  hs_opts o;
  if (!merge_opts(opts, &o)) return HS_ERR_INVALID;
  if (o.alpha_trace || o.restart_iters) {
    set_error("the BiCGStab trace is read back to the host: not available in the asynchronous form");
    return HS_ERR_INVALID;
  }
  if (res_dev && !aligned(res_dev, 8)) {
    set_error("res must be an 8-byte aligned device pointer");
    return HS_ERR_INVALID;
  }
  hs_status s = check_solve(A, dt, b, x, tol, maxit, ws, ws_bytes, which, o);
  if (s != HS_OK) return s;
  SolveArgs a;
  a.A = A;
  a.dtype = dt;
  a.b = b;
  a.x = x;
  a.tol = tol;
  a.maxit = maxit;
  a.o = o;
  a.ws = (char*)ws;
  a.ws_bytes = ws_bytes;
  a.stream = (cudaStream_t)stream;
  a.async_dev = true;
  a.res_dev = res_dev;
  a.hist_dev = hist_dev;
  cudaError_t e = cudaGetLastError();  // clear stale errors from unrelated work
  (void)e;
  hs_result scratch;
  fill_res(&scratch);
  return run(a, &scratch, nullptr);
}

}  // namespace hs

using namespace hs;

extern "C" {

const char* hs_last_error(void) { return g_err; }
const char* hs_version(void) { return "hsolve 0.1 (sm_103a)"; }
int hs_last_staging(void) { return g_last_staging; }

hs_status hs_diag_wait_timeout(int kind, double timeout_s, void* stream) {
  if (kind < 0 || kind > 3) {
    set_error("kind must be 0 (grid barrier), 1 (Gauss-Seidel tile wait), 2 (27-point ring wait) or 3 (27-point "
              "plane waits)");
    return HS_ERR_INVALID;
  }
  if (!(timeout_s > 0.0) || timeout_s > 10.0) {
    set_error("timeout_s must lie in (0, 10]");
    return HS_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  char* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, 4096);
  if (e != cudaSuccess) return cuda_fail(e, "diagnostic buffer");
  // control block, then zeroed words: barrier partials / flags / progress
  Common cm{reinterpret_cast<Ctrl*>(buf), reinterpret_cast<double*>(buf + 512), nullptr};
  hs_opts o = default_opts();
  o.timeout_s = timeout_s;
  hs_status s = HS_OK;
  e = cudaMemsetAsync(buf, 0, 4096, st);
  if (e != cudaSuccess) s = cuda_fail(e, "diagnostic buffer");
  if (s == HS_OK) s = init_ctrl(cm, o, st);
  if (s == HS_OK) {
    if (kind == 0) s = diag_team_wait(cm.ctrl, cm.partials, st);
    else if (kind == 1) s = diag_gs_wait(cm.ctrl, reinterpret_cast<const unsigned*>(buf + 1024), st);
    else if (kind == 2) s = diag_gs27_wait(cm.ctrl, reinterpret_cast<const unsigned long long*>(buf + 1024), st);
    else s = diag_gs27p_wait(cm.ctrl, reinterpret_cast<unsigned long long*>(buf + 1024), st);
  }
  int status = 0;
  if (s == HS_OK) {
    e = cudaMemcpyAsync(&status, &cm.ctrl->status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_fail(e, "diagnostic wait");
  }
  cudaError_t ef = cudaFree(buf);
  if (s != HS_OK) return s;
  if (ef != cudaSuccess) return cuda_fail(ef, "diagnostic buffer");
  if (status == DS_TIMEOUT) {
    set_error("the wait gave up after %g s, as designed", timeout_s);
    return HS_ERR_TIMEOUT;
  }
  return HS_OK;
}

hs_status hs_grid_create(int ndim, const int64_t n[3], hs_grid** out) {
  if (!out) { set_error("out is NULL"); return HS_ERR_INVALID; }
  *out = nullptr;
  if (ndim < 1 || ndim > 3 || !n) { set_error("ndim must be 1, 2 or 3"); return HS_ERR_INVALID; }
  int64_t N = 1;
  for (int d = 0; d < ndim; d++) {
    if (n[d] < 1 || n[d] > (int64_t)1 << 30) { set_error("grid extent n[%d] out of range", d); return HS_ERR_INVALID; }
    N *= n[d];
    if (N >= ((int64_t)1 << 31)) { set_error("grid too large (N must be < 2^31)"); return HS_ERR_INVALID; }
  }
  hs_grid* g = new (std::nothrow) hs_grid;
  if (!g) { set_error("out of host memory"); return HS_ERR_INVALID; }
  g->ndim = ndim;
  for (int d = 0; d < 3; d++) g->n[d] = d < ndim ? n[d] : 1;
  *out = g;
  return HS_OK;
}

void hs_grid_destroy(hs_grid* g) { delete g; }

static hs_status make_op(const hs_grid* g, int kind, const double* beta, const void* k, int kdt, hs_op** out) {
  if (!out) { set_error("out is NULL"); return HS_ERR_INVALID; }
  *out = nullptr;
  if (!g) { set_error("grid is NULL"); return HS_ERR_INVALID; }
  hs_op* A = new (std::nothrow) hs_op;
  if (!A) { set_error("out of host memory"); return HS_ERR_INVALID; }
  memset(A, 0, sizeof(*A));
  A->ndim = g->ndim;
  A->kind = kind;
  for (int d = 0; d < 3; d++) {
    A->n[d] = g->n[d];
    A->h[d] = d < g->ndim ? 1.0 / (double)(g->n[d] + 1) : 1.0;
    A->beta[d] = (beta && d < g->ndim) ? beta[d] : 0.0;
  }
  A->k = k;
  A->kdt = kdt;
  *out = A;
  return HS_OK;
}

hs_status hs_op_laplacian(const hs_grid* g, hs_op** out) { return make_op(g, KIND_LAPLACIAN, nullptr, nullptr, 0, out); }

hs_status hs_op_hpcg(const hs_grid* g, int points, hs_op** out) {
  if (points != 7 && points != 27) { set_error("points must be 7 or 27"); return HS_ERR_INVALID; }
  if (points == 27 && g && g->ndim != 3) { set_error("the 27-point system needs a 3-D grid"); return HS_ERR_INVALID; }
  return make_op(g, points == 7 ? KIND_HPCG7 : KIND_HPCG27, nullptr, nullptr, 0, out);
}

hs_status hs_op_convdiff_upwind(const hs_grid* g, const double beta[3], hs_op** out) {
  if (!beta) { set_error("beta is NULL"); return HS_ERR_INVALID; }
  if (g)
    for (int d = 0; d < g->ndim; d++)
      if (!(beta[d] >= 0.0) || !isfinite(beta[d])) {
        set_error("beta[%d] must be finite and >= 0 (first-order upwind)", d);
        return HS_ERR_INVALID;
      }
  return make_op(g, KIND_UPWIND, beta, nullptr, 0, out);
}

hs_status hs_op_diffusion(const hs_grid* g, hs_dtype kdt, const void* k_dev, hs_op** out) {
  if (!k_dev) { set_error("k is NULL"); return HS_ERR_INVALID; }
  if (kdt != HS_F64 && kdt != HS_F32) { set_error("k dtype must be HS_F64 or HS_F32"); return HS_ERR_INVALID; }
  if (!aligned(k_dev, 16)) { set_error("k must be 16-byte aligned"); return HS_ERR_INVALID; }
  return make_op(g, KIND_DIFFUSION, nullptr, k_dev, kdt, out);
}

void hs_op_destroy(hs_op* op) { delete op; }

int64_t hs_op_size(const hs_op* op) { return op ? op->n[0] * op->n[1] * op->n[2] : 0; }

hs_status hs_spmv(const hs_op* A, hs_dtype dtype, const void* x, void* y, void* stream) {
  NvtxRange range("hs_spmv");
  if (!A || !x || !y) { set_error("NULL argument"); return HS_ERR_INVALID; }
  if (dtype != HS_F64 && dtype != HS_F32) { set_error("bad dtype"); return HS_ERR_INVALID; }
  if (x == y) { set_error("x and y must not alias"); return HS_ERR_INVALID; }
  if (!aligned(x, 16) || !aligned(y, 16)) { set_error("x and y must be 16-byte aligned"); return HS_ERR_INVALID; }
  return run_spmv(A, dtype, x, y, (cudaStream_t)stream);
}

hs_status hs_residual(const hs_op* A, hs_dtype dtype, const void* b, const void* x, void* r, void* stream) {
  NvtxRange range("hs_residual");
  if (!A || !b || !x || !r) { set_error("NULL argument"); return HS_ERR_INVALID; }
  if (dtype != HS_F64 && dtype != HS_F32) { set_error("bad dtype"); return HS_ERR_INVALID; }
  if (r == x || r == b) { set_error("r must not alias b or x"); return HS_ERR_INVALID; }
  if (!aligned(x, 16) || !aligned(b, 16) || !aligned(r, 16)) { set_error("vectors must be 16-byte aligned"); return HS_ERR_INVALID; }
  return hs::run_residual_plain(A, dtype, b, x, r, (cudaStream_t)stream);
}

hs_status hs_workspace_size(const hs_op* A, hs_solver solver, hs_dtype dtype, const hs_opts* opts, int maxit,
                            size_t* bytes) {
  if (!A || !bytes) { set_error("NULL argument"); return HS_ERR_INVALID; }
  if (dtype != HS_F64 && dtype != HS_F32) { set_error("bad dtype"); return HS_ERR_INVALID; }
  if (solver < HS_SOLVER_JACOBI || solver > HS_SOLVER_CG_NB) { set_error("bad solver"); return HS_ERR_INVALID; }
  if (solver == HS_SOLVER_MIXED && dtype != HS_F64) { set_error("mixed precision takes FP64 b and x"); return HS_ERR_INVALID; }
  if (maxit < 0) { set_error("maxit must be >= 0"); return HS_ERR_INVALID; }
  hs_opts o;
  if (!merge_opts(opts, &o)) return HS_ERR_INVALID;
  *bytes = ws_need(A, solver, dtype, o, maxit);
  return HS_OK;
}

hs_status hs_solve_mixed(const hs_op* A, const double* b, double* x, double tol, int maxit, const hs_opts* opts,
                         void* ws, size_t ws_bytes, void* stream, hs_result* res, double* hist) {
  return solve_common(run_mixed, HS_SOLVER_MIXED, A, HS_F64, b, x, tol, maxit, opts, ws, ws_bytes, stream, res,
                      hist);
}

hs_status hs_jacobi(const hs_op* A, hs_dtype dtype, const void* b, void* x, double tol, int maxit,
                    const hs_opts* opts, void* ws, size_t ws_bytes, void* stream, hs_result* res, double* hist) {
  return solve_common(run_jacobi, HS_SOLVER_JACOBI, A, dtype, b, x, tol, maxit, opts, ws, ws_bytes, stream, res,
                      hist);
}

hs_status hs_gauss_seidel(const hs_op* A, hs_dtype dtype, const void* b, void* x, double tol, int maxit,
                          const hs_opts* opts, void* ws, size_t ws_bytes, void* stream, hs_result* res,
                          double* hist) {
  return solve_common(run_gauss_seidel, HS_SOLVER_GAUSS_SEIDEL, A, dtype, b, x, tol, maxit, opts, ws, ws_bytes,
                      stream, res, hist);
}

hs_status hs_cg(const hs_op* A, hs_dtype dtype, const void* b, void* x, double tol, int maxit, const hs_opts* opts,
                void* ws, size_t ws_bytes, void* stream, hs_result* res, double* hist) {
  if (A && opkind_of(A) == OP_NONSYM) {
    set_error("CG needs a symmetric operator (Laplacian or diffusion)");
    if (res) { fill_res(res); }
    return HS_ERR_INVALID;
  }
  return solve_common(run_cg, HS_SOLVER_CG, A, dtype, b, x, tol, maxit, opts, ws, ws_bytes, stream, res, hist);
}

hs_status hs_cg_nb(const hs_op* A, hs_dtype dtype, const void* b, void* x, double tol, int maxit,
                   const hs_opts* opts, void* ws, size_t ws_bytes, void* stream, hs_result* res, double* hist) {
  if (A && opkind_of(A) == OP_NONSYM) {
    set_error("CG-NB needs a symmetric operator (Laplacian or diffusion)");
    if (res) { fill_res(res); }
    return HS_ERR_INVALID;
  }
  return solve_common(run_cg_nb, HS_SOLVER_CG_NB, A, dtype, b, x, tol, maxit, opts, ws, ws_bytes, stream, res,
                      hist);
}

hs_status hs_bicgstab(const hs_op* A, hs_dtype dtype, const void* b, void* x, double tol, int maxit,
                      const hs_opts* opts, void* ws, size_t ws_bytes, void* stream, hs_result* res, double* hist) {
  return solve_common(run_bicgstab, HS_SOLVER_BICGSTAB, A, dtype, b, x, tol, maxit, opts, ws, ws_bytes, stream, res,
                      hist);
}

hs_status hs_jacobi_async(const hs_op* A, hs_dtype dtype, const void* b, void* x, double tol, int maxit,
                          const hs_opts* opts, void* ws, size_t ws_bytes, void* stream, hs_result* res_dev,
                          double* hist_dev) {
  return solve_async(run_jacobi, HS_SOLVER_JACOBI, A, dtype, b, x, tol, maxit, opts, ws, ws_bytes, stream, res_dev,
                     hist_dev);
}

hs_status hs_gauss_seidel_async(const hs_op* A, hs_dtype dtype, const void* b, void* x, double tol, int maxit,
                                const hs_opts* opts, void* ws, size_t ws_bytes, void* stream, hs_result* res_dev,
                                double* hist_dev) {
  return solve_async(run_gauss_seidel, HS_SOLVER_GAUSS_SEIDEL, A, dtype, b, x, tol, maxit, opts, ws, ws_bytes, stream,
                     res_dev, hist_dev);
}

hs_status hs_cg_async(const hs_op* A, hs_dtype dtype, const void* b, void* x, double tol, int maxit,
                      const hs_opts* opts, void* ws, size_t ws_bytes, void* stream, hs_result* res_dev,
                      double* hist_dev) {
  if (A && opkind_of(A) == OP_NONSYM) {
    set_error("CG needs a symmetric operator (Laplacian or diffusion)");
    return HS_ERR_INVALID;
  }
  return solve_async(run_cg, HS_SOLVER_CG, A, dtype, b, x, tol, maxit, opts, ws, ws_bytes, stream, res_dev, hist_dev);
}

hs_status hs_bicgstab_async(const hs_op* A, hs_dtype dtype, const void* b, void* x, double tol, int maxit,
                            const hs_opts* opts, void* ws, size_t ws_bytes, void* stream, hs_result* res_dev,
                            double* hist_dev) {
  return solve_async(run_bicgstab, HS_SOLVER_BICGSTAB, A, dtype, b, x, tol, maxit, opts, ws, ws_bytes, stream,
                     res_dev, hist_dev);
}

}  // extern "C"
