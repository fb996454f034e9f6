/*
 * hsolve.h -- C ABI of libhsolve, a single-GPU (sm_103a) library of the four
 * classical iterative methods studied in Martinez-Ferrer, Arslan & Beltran,
 * "Improving the performance of classical linear algebra iterative methods
 * via hybrid parallelism" (arXiv 2305.05988): Jacobi, Gauss-Seidel,
 * conjugate gradient and BiCGStab, applied matrix-free to structured-grid
 * finite-difference operators.
 *
 * The paper solves A x = b with a known sparse A arising from a centred
 * stencil on a structured mesh (section 3.1, section 4.1).  Here A is never
 * stored: it is one of three stencil operators on a grid of n_x [* n_y
 * [* n_z]] interior nodes, spacing h_d = 1/(n_d + 1), homogeneous Dirichlet
 * boundary (zero ghost values):
 *   - Laplacian   A = -Delta_h                (5-point 2-D, 7-point 3-D)
 *   - upwind      -Delta u + beta . grad u, beta_d >= 0, first-order upwind
 *   - diffusion   -div(k grad u), harmonic-mean face coefficients, a
 *                 boundary face using the cell's own k.
 *
 * Conventions shared by every entry point
 *   - Vectors are dense, contiguous, lexicographic idx = i + n_x (j + n_y k)
 *     (i fastest), of length N = prod n_d, in DEVICE memory, 16-byte
 *     aligned, owned by the caller; the library never frees or retains them.
 *   - dtype HS_F64 means IEEE binary64 elements, HS_F32 binary32.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Every call is stream-ordered; the solver entry points
 *     synchronise `stream` before returning because they report a host-side
 *     result.
 *   - Solvers take a caller-allocated device workspace of at least
 *     hs_workspace_size() bytes (256-byte aligned); the library allocates
 *     no device memory per call.  Workspaces must not be shared by calls
 *     that may overlap on the GPU.
 *   - Errors are returned, never thrown or trapped on the device.  After a
 *     non-OK status hs_last_error() gives a message (thread-local).
 *   - Every device-side wait (grid barrier, wavefront flag) is bounded; a
 *     wait that runs out ends the kernel with HS_ERR_TIMEOUT instead of
 *     hanging.
 */
#ifndef HSOLVE_H
#define HSOLVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HS_OK = 0,               /* converged, or ran the requested sweeps            */
    HS_NOT_CONVERGED = 1,    /* maxit reached; x holds the last iterate           */
    HS_ERR_INVALID = -1,     /* bad argument (null pointer, shape, dtype, ...)    */
    HS_ERR_CUDA = -2,        /* a CUDA runtime call failed                         */
    HS_ERR_BREAKDOWN = -3,   /* a Krylov denominator vanished (e.g. p.Ap <= 0)     */
    HS_ERR_NONFINITE = -4,   /* NaN or Inf appeared in a reduction                 */
    HS_ERR_TIMEOUT = -5,     /* a bounded device-side wait ran out                 */
    HS_ERR_WORKSPACE = -6,   /* workspace missing, misaligned or too small         */
    HS_ERR_BOUNDS = -7       /* debug builds only: a kernel computed an index
                                outside a vector (the access was skipped)         */
} hs_status;

typedef enum { HS_F64 = 0, HS_F32 = 1 } hs_dtype;

typedef enum {
    HS_SOLVER_JACOBI = 0,
    HS_SOLVER_GAUSS_SEIDEL = 1,
    HS_SOLVER_CG = 2,
    HS_SOLVER_BICGSTAB = 3,
    HS_SOLVER_MIXED = 4,     /* hs_solve_mixed (dtype HS_F64) */
    HS_SOLVER_CG_NB = 5      /* hs_cg_nb */
} hs_solver;

typedef enum { HS_GS_FORWARD = 0, HS_GS_BACKWARD = 1, HS_GS_SYMMETRIC = 2 } hs_gs_mode;

typedef struct hs_grid hs_grid;   /* opaque, library-owned */
typedef struct hs_op hs_op;       /* opaque, library-owned */

/*
 * Solver options.  Set struct_size = sizeof(hs_opts); fields beyond a
 * caller's struct_size take their defaults.  Pass NULL for all defaults.
 */
typedef struct {
    size_t struct_size;
    int gs_mode;            /* hs_gs_mode; default HS_GS_FORWARD (one sweep per
                               iteration; HS_GS_SYMMETRIC is the paper's
                               symmetric GS, section 3.1)                        */
    int check_every;        /* GS with tol > 0: test the residual every this many
                               iterations (default 1)                           */
    double restart_eps;     /* BiCGStab restart threshold eps' on sqrt|alpha_n|,
                               Algorithm 2 (default 1e-5; 0 disables)           */
    int true_residual;      /* 1 (default): compute ||b - A x|| / ||b|| of the
                               returned x into hs_result.true_rel_res           */
    double timeout_s;       /* bound on any single device-side wait, seconds
                               (default 2.0)                                     */
    double inner_tol;       /* mixed precision: inner relative tolerance (1e-5) */
    int inner_solver;       /* mixed precision: HS_SOLVER_CG or _BICGSTAB (CG)  */
    int inner_maxit;        /* mixed precision: inner iteration cap (10000)     */
    int use_graph;          /* batched solver: replay one captured CUDA graph
                               (default 1; needs a non-default stream)          */
    int tile_rows;          /* stencil tiles of the Jacobi / CG / BiCGStab /
                               mixed solvers: rows of 32 nodes per tile = warps
                               per block, 4 to 16 (other values: the built-in
                               heuristic, 8 rows on 3-D grids)                 */
    int tile_planes;        /* z planes per work item of those tiles; 0 = the
                               built-in cost model                             */
    int max_blocks;         /* cap on the persistent grid (blocks); 0 = all
                               co-resident blocks                               */
    int paper_order;        /* 1: the statement order printed in Algorithms 1-2
                               (convergence tested at the top of the next
                               iteration / after omega, then the final step
                               x = x_l + alpha_l p_l (CG-NB) or
                               x = x_l + omega_l s_l (BiCGStab), which returns
                               the iterate one step beyond the converged one);
                               0 (default): test right after each residual
                               update and return that iterate                   */
    int sweeps_per_pass;    /* Jacobi: sweeps applied per pass over the grid
                               (temporal blocking, 1..4; default 1).  Used for
                               constant-coefficient 3-D 7-point operators with
                               tol = 0; the iterates are bitwise those of single
                               sweeps.  Other cases run one sweep per pass.     */
    double *alpha_trace;    /* BiCGStab diagnostics (hs_bicgstab only): host
                               array of maxit + 1 doubles, may be NULL.  Entry
                               k receives r_k . r' after iteration k, the value
                               whose square root Algorithm 2's restart test
                               compares with restart_eps (entry 0: r_0 . r').
                               Entries beyond res.iters are left untouched.   */
    int *restart_iters;     /* BiCGStab diagnostics: host array of maxit ints,
                               may be NULL; receives the iterations after which
                               a restart was taken, in order (res.restarts of
                               them).                                          */
    int staging;            /* FP32 CG on a 3-D diffusion operator (hs_cg with
                               HS_F32, and the inner CG of hs_solve_mixed):
                               0 (default) the register-prefetch tile engine
                               on stored FP32 coefficient arrays (16 B of
                               operator data per node, the fastest measured);
                               1 the stencil planes staged in shared memory by
                               TMA and the face coefficients formed from k
                               (4 B per node; 3-D, n_x a multiple of 4,
                               n_x >= 40, n_y >= 10, n_z >= 3, else
                               HS_ERR_INVALID)                                  */
    int inner_fixed_tol;    /* mixed precision (hs_solve_mixed and the mixed
                               batch): 0 (default) a refinement step whose
                               FP64 relative residual rel_k is already near
                               tol stops its inner solve early, at the inner
                               relative tolerance max(inner_tol,
                               0.5 tol / rel_k), which is all the step needs
                               to reach tol; 1: every inner solve runs to
                               inner_tol                                       */
    int gs_schedule;        /* lexicographic Gauss-Seidel: 0 (default) on
                               3-D grids the pencil schedule for batches of
                               four or more sweeps of one direction on
                               constant-coefficient operators with between
                               12 pencils per SM and one pencil per resident
                               warp, the tile schedule otherwise; on 1-/2-D
                               grids whose iterate fits shared memory, for
                               such pipelined batches one thread-block
                               cluster (8 CTAs, rows split over them,
                               distributed shared memory), else (single
                               sweeps, symmetric, max_blocks = 1, fewer than
                               16 rows) one block; 1 the tile schedule on
                               every grid (tiles of
                               32 x 8 x 8 or 32 x 16 x 16 nodes swept along
                               point hyperplanes in shared memory, ordered by
                               per-tile sweep counts); 2 the pencil schedule
                               (one warp per 8 x 4 x-lines streaming two nodes
                               per substep, neighbour lines by warp shuffles,
                               ordered by per-pencil progress counts; 3-D
                               constant-coefficient 7-point operators only:
                               Laplacian, upwind, HPCG 7-point; else
                               HS_ERR_INVALID); 3 one thread-block cluster
                               (2-D grids of at least 16 rows that fit, no
                               max_blocks; else HS_ERR_INVALID).  The HPCG
                               27-point operator: 0 the plane-lagged schedule
                               for single sweeps and the symmetric method when
                               an x-y plane fits 200 KB of shared memory, the
                               hyperplane schedule otherwise; 1 the hyperplane
                               schedule (one grid-wide step per point
                               hyperplane i + 2j + 4k, sweeps of one direction
                               pipelined); 2 the plane-lagged schedule (whole
                               z planes per block in shared memory, planes
                               pipelined four in-plane steps apart; the plane
                               must fit 200 KB with min(n_y, ceil(n_x / 2)) <=
                               112, else HS_ERR_INVALID); 3
                               HS_ERR_INVALID.  All give bitwise the same
                               iterates.                                       */
} hs_opts;

typedef struct {
    int iters;              /* iterations (sweeps for Jacobi / forward or backward
                               GS, forward+backward pairs for symmetric GS)     */
    int status;             /* hs_status of the solve                            */
    double rel_res;         /* last recursive relative residual (Krylov) or the
                               relative residual of the returned iterate        */
    double true_rel_res;    /* ||b - A x|| / ||b|| of the returned x, or -1      */
    int restarts;           /* BiCGStab restarts taken                           */
    int outer;              /* mixed precision: refinement steps taken           */
    long long inner_iters;  /* mixed precision: total inner iterations           */
} hs_result;

/* ---- grids and operators (host objects; no device memory is allocated) --- */

/* ndim in {1, 2, 3}; n[d] >= 1 for d < ndim (entries beyond ndim ignored).
 * N = prod n_d must be below 2^31.  Returns HS_ERR_INVALID otherwise. */
hs_status hs_grid_create(int ndim, const int64_t n[3], hs_grid **out);
void hs_grid_destroy(hs_grid *g);

/* Operators keep a copy of the grid; the grid may be destroyed afterwards. */
hs_status hs_op_laplacian(const hs_grid *g, hs_op **out);
/* The benchmark system of section 4.1 (HPCG's generated matrix, unscaled):
 * diagonal 27 and -1 for each of the 6 face neighbours (points = 7) or the 26
 * neighbours of the 3x3x3 box (points = 27, 3-D grids only) inside the grid.
 * The paper solves it with b = A 1 (exact solution x = 1) from x0 = 0 to an
 * absolute residual of 1e-6.  The coefficients are the reading that fits the
 * paper's printed iteration counts.  The 27-point operator supports SpMV,
 * residual, Jacobi, CG, CG-NB, BiCGStab, mixed precision and lexicographic
 * Gauss-Seidel (one step per point hyperplane i + 2j + 4k, so a
 * sweep takes nx + 2 ny + 4 nz steps); the batched solver returns
 * HS_ERR_INVALID for it.
 * HS_ERR_INVALID: points not 7 or 27, a 27-point operator on a 1-/2-D grid. */
hs_status hs_op_hpcg(const hs_grid *g, int points, hs_op **out);

/* beta[d] >= 0 and finite for d < ndim (first-order upwind). */
hs_status hs_op_convdiff_upwind(const hs_grid *g, const double beta[3], hs_op **out);
/* k_dev: device array of N coefficients (> 0) of type kdt, BORROWED: it must
 * stay valid and unchanged for the operator's lifetime. */
hs_status hs_op_diffusion(const hs_grid *g, hs_dtype kdt, const void *k_dev, hs_op **out);
void hs_op_destroy(hs_op *op);
/* Number of unknowns N of an operator (0 for NULL). */
int64_t hs_op_size(const hs_op *op);

/* ---- single operator application --------------------------------------- */

/* y = A x (the sparse matrix-vector product of section 3.1, matrix-free).
 * x, y: device vectors of N elements of `dtype`; must not alias. */
hs_status hs_spmv(const hs_op *A, hs_dtype dtype, const void *x, void *y, void *stream);

/* r = b - A x (device vectors of N elements of dtype; r must not alias b or x). */
hs_status hs_residual(const hs_op *A, hs_dtype dtype, const void *b, const void *x, void *r,
                      void *stream);

/* ---- solvers --------------------------------------------------------------
 * Common arguments:
 *   b        device right-hand side (N elements of dtype)
 *   x        device initial guess on entry, solution on exit (N elements)
 *   tol      relative-residual target ||b - A x|| / ||b|| (Krylov: recursive
 *            residual).  tol == 0 runs exactly maxit iterations (Jacobi/GS).
 *   maxit    iteration cap (>= 0)
 *   opts     NULL for defaults
 *   ws       device workspace, ws_bytes >= hs_workspace_size(...)
 *   res      host hs_result, may be NULL
 *   hist     host array of maxit + 1 doubles, may be NULL: hist[k] is the
 *            relative residual after k iterations (entries beyond res.iters
 *            are left untouched).  Jacobi / GS record it only when tol > 0.
 * A zero right-hand side returns x = 0 after 0 iterations.
 */
hs_status hs_workspace_size(const hs_op *A, hs_solver solver, hs_dtype dtype, const hs_opts *opts,
                            int maxit, size_t *bytes);

/* Jacobi (section 3.1): x_i <- (b_i - sum_{j != i} a_ij x_j) / a_ii, undamped,
 * out of place.  With tol > 0 the residual of each iterate is fused into the
 * next sweep and the first iterate x_k with relative residual <= tol is
 * returned (iters = k). */
hs_status hs_jacobi(const hs_op *A, hs_dtype dtype, const void *b, void *x, double tol, int maxit,
                    const hs_opts *opts, void *ws, size_t ws_bytes, void *stream, hs_result *res,
                    double *hist);

/* Gauss-Seidel (section 3.1), exactly lexicographic: every update uses the
 * entries already updated in the same sweep (forward: idx ascending,
 * backward: descending; symmetric = forward then backward).  No recolouring:
 * the result equals the sequential sweep up to rounding.  x is updated in
 * place.  Performance: sweeps of one direction between residual checks
 * (opts->check_every with tol > 0, all maxit sweeps with tol == 0) overlap
 * when there are four or more of them; single sweeps and the symmetric method
 * run one after another.  The 27-point HPCG operator takes one step per point
 * hyperplane (nx + 2 ny + 4 nz per sweep).  opts->max_blocks caps the grid.
 * The workspace holds b / a_ii and the schedule's tables
 * (hs_workspace_size). */
hs_status hs_gauss_seidel(const hs_op *A, hs_dtype dtype, const void *b, void *x, double tol,
                          int maxit, const hs_opts *opts, void *ws, size_t ws_bytes, void *stream,
                          hs_result *res, double *hist);

/* Conjugate gradient, the classical method HPCCG runs (section 3.2), with the
 * stencil, vector updates and dot products fused into two passes per
 * iteration.  A must be symmetric positive definite (Laplacian, diffusion). */
hs_status hs_cg(const hs_op *A, hs_dtype dtype, const void *b, void *x, double tol, int maxit,
                const hs_opts *opts, void *ws, size_t ws_bytes, void *stream, hs_result *res,
                double *hist);

/* CG-NB, the paper's nonblocking CG (section 3.2, Algorithm 1): the SpMV is
 * applied to r_j and A p_j = A r_j + beta_j A p_j-1 follows by recurrence.
 * One fused pass and ONE reduce-barrier per iteration: the denominator
 * (A p_j).p_j is expanded as r_j.A r_j + 2 beta_j r_j.A p_j-1
 * + beta_j^2 (A p_j-1).p_j-1 (exact for symmetric A), so r.r, r.A r and
 * r.A p_j-1 are reduced together before beta_j is known.
 * A must be symmetric positive definite.  x is updated as x_j-1 + alpha_j-1
 * p_j-1 (Algorithm 1's x_j-1 + c (p_j - r_j) with c (p_j - r_j) = alpha_j-1
 * p_j-1).  Workspace: hs_workspace_size(A, HS_SOLVER_CG_NB, ...). */
hs_status hs_cg_nb(const hs_op *A, hs_dtype dtype, const void *b, void *x, double tol, int maxit,
                   const hs_opts *opts, void *ws, size_t ws_bytes, void *stream, hs_result *res,
                   double *hist);

/* BiCGStab with the shadow residual r' = r0/||r0|| and the restart rule of
 * Algorithm 2 (restart when sqrt|alpha_n| < restart_eps: p = r, r' = r/||r||),
 * classical statement order (convergence tested after each residual update);
 * opts.paper_order = 1 gives Algorithm 2's order (BiCGStab-B1: test on the
 * previous residual after omega, then the final step x = x_l + omega_l s_l). */
hs_status hs_bicgstab(const hs_op *A, hs_dtype dtype, const void *b, void *x, double tol,
                      int maxit, const hs_opts *opts, void *ws, size_t ws_bytes, void *stream,
                      hs_result *res, double *hist);

/* Asynchronous forms of the four solvers, for CUDA-graph capture: the same
 * arguments, validation and workspace as hs_jacobi / hs_gauss_seidel / hs_cg /
 * hs_bicgstab, but nothing on the host waits for the GPU.  The call validates
 * its arguments (returning HS_ERR_INVALID / HS_ERR_WORKSPACE at once, as the
 * synchronous calls do), enqueues the solve on `stream` and returns HS_OK;
 * the solver's outcome is written by a kernel at the end of the work into
 * res_dev (DEVICE memory, one hs_result, 8-byte aligned, may be NULL) and the
 * residual history into hist_dev (DEVICE memory, maxit + 1 doubles, may be
 * NULL; entries up to res.iters are written, as in the synchronous form).
 * Every step of these calls is stream-ordered (kernel launches and
 * device-to-device copies only), so a call can be captured in a CUDA graph
 * and the graph replayed with new contents of b and x; the workspace, vectors
 * and result buffers must then stay allocated.  Not available: the BiCGStab
 * trace options (alpha_trace, restart_iters: HS_ERR_INVALID) and the debug
 * build's bounds report, which synchronises. */
hs_status hs_jacobi_async(const hs_op *A, hs_dtype dtype, const void *b, void *x, double tol, int maxit,
                          const hs_opts *opts, void *ws, size_t ws_bytes, void *stream, hs_result *res_dev,
                          double *hist_dev);
hs_status hs_gauss_seidel_async(const hs_op *A, hs_dtype dtype, const void *b, void *x, double tol,
                                int maxit, const hs_opts *opts, void *ws, size_t ws_bytes, void *stream,
                                hs_result *res_dev, double *hist_dev);
hs_status hs_cg_async(const hs_op *A, hs_dtype dtype, const void *b, void *x, double tol, int maxit,
                      const hs_opts *opts, void *ws, size_t ws_bytes, void *stream, hs_result *res_dev,
                      double *hist_dev);
hs_status hs_bicgstab_async(const hs_op *A, hs_dtype dtype, const void *b, void *x, double tol,
                            int maxit, const hs_opts *opts, void *ws, size_t ws_bytes, void *stream,
                            hs_result *res_dev, double *hist_dev);

/* Mixed-precision iterative refinement.  Not in the paper (which is FP64
 * throughout); it gets the FP64 answer of A x = b at FP32 cost on a GPU whose
 * FP32 pipe is 64x its FP64 pipe.  Each refinement step computes the FP64
 * residual r = b - A x and its relative norm on the GPU (stop when <= tol),
 * solves A d = r/||r|| with CG (opts.inner_solver = HS_SOLVER_CG, symmetric
 * operators) or BiCGStab on FP32 vectors and FP32 coefficients with dot
 * products accumulated in FP64, to the relative tolerance opts.inner_tol
 * (default 1e-5) or opts.inner_maxit iterations, and updates x += ||r|| d in
 * FP64.  b, x: FP64 device vectors.  maxit bounds the refinement steps.
 * res.iters = res.outer = refinement steps, res.inner_iters = their total
 * inner iterations, res.rel_res = res.true_rel_res = FP64 relative residual
 * of the returned x; hist[k] = that residual after k steps (maxit + 1 doubles).
 * Workspace: hs_workspace_size(A, HS_SOLVER_MIXED, HS_F64, opts, maxit, &n). */
hs_status hs_solve_mixed(const hs_op *A, const double *b, double *x, double tol, int maxit,
                         const hs_opts *opts, void *ws, size_t ws_bytes, void *stream,
                         hs_result *res, double *hist);

/* Adjoint gradient through the diffusion solve.  Not in the paper: it
 * differentiates a loss L(u) with A(k) u = f for inverse problems.  Given the
 * forward solution u and the adjoint lam solving A^T lam = dL/du (A is
 * symmetric, so lam comes from hs_cg with right-hand side dL/du), writes
 *   g_i = dL/dlog k_i = -k_i sum_{faces f of i} dkappa_f/dk_i
 *                        (lam_i - lam_j)(u_i - u_j) / h_d^2,
 * dkappa_f/dk_i = 2 k_j^2 / (k_i + k_j)^2 for an interior face and 1 for a
 * boundary face (lam_j = u_j = 0).  dL/df is lam itself.  u, lam, g: FP64
 * device vectors of N elements; g must not alias u or lam.  A must be a
 * diffusion operator (HS_ERR_INVALID otherwise). */
hs_status hs_diffusion_grad_logk(const hs_op *A, const double *u, const double *lam, double *g,
                                 void *stream);

/* k_i = exp(logk_i) for i < n: the diffusion coefficient field from the
 * log-coefficients in which hs_diffusion_grad_logk differentiates (the inverse
 * problem parametrises k > 0 by log k; not in the paper).  logk, k: FP64
 * device vectors of n elements; k may be logk itself (in place) but must not
 * overlap it otherwise.  exp overflows to +inf above log k = 709.78 and
 * underflows to 0 below about -745; neither is a valid coefficient for
 * hs_op_diffusion, so callers keep log k well inside that range.
 * Asynchronous on `stream`.  HS_ERR_INVALID: n < 0, NULL vectors with n > 0,
 * partial overlap. */
hs_status hs_exp_logk(const double *logk, double *k, int64_t n, void *stream);

/* ---- conjugate gradient without any allocation --------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory themselves -- for example a plug-in
 * inside a host application that hands out all GPU memory through its own
 * pool and forbids foreign cudaMalloc calls, or a latency-critical path that
 * must not enter an allocator.  hs_cg_static runs exactly the solver of
 * hs_cg, but its workspace is a fixed array of HS_STATIC_SCRATCH_BYTES bytes
 * inside the library's device image (held by every GPU that loads the
 * library until the process exits), so the call allocates nothing; the
 * caller still owns b and x.
 *   - Problems whose CG workspace (hs_workspace_size with HS_SOLVER_CG, the
 *     same dtype and maxit) exceeds HS_STATIC_SCRATCH_BYTES are rejected with
 *     HS_ERR_INVALID and a message naming both sizes.  With FP64 and a
 *     constant-coefficient operator that is about 500 k unknowns.
 *   - The first call on a device, with that device current, looks up the
 *     array's device address (cudaGetSymbolAddress) and keeps it: make that
 *     first call before any stream capture on that device.  Resetting the
 *     device (cudaDeviceReset) while the library is loaded is not supported.
 *   - `stream` must belong to the current device (HS_ERR_INVALID otherwise):
 *     the kept address is that device's.
 *   - All calls on a device share the one array and it keeps the previous
 *     call's contents; the solver initialises what it reads first.  Calls that
 *     may overlap on the GPU (other streams, other host threads) race on the
 *     array and must be serialised by the caller.
 * Arguments and results are those of hs_cg. */
#define HS_STATIC_SCRATCH_BYTES (16u << 20)
hs_status hs_cg_static(const hs_op *A, hs_dtype dtype, const void *b, void *x, double tol, int maxit,
                       const hs_opts *opts, void *stream, hs_result *res, double *hist);

/* ---- batched solves -------------------------------------------------------
 * Many independent systems (grids of any size and dimension, CG or BiCGStab
 * each) solved by ONE persistent cooperative kernel, replayed as a CUDA graph.
 * Not in the paper (which solves one system per run); it keeps the GPU full
 * when each system alone is too small to.  The library splits the grid into
 * teams: a system whose estimated work (unknowns x iterations) exceeds the
 * planned makespan gets a team of blocks of its own; the other systems form a
 * queue, largest first, that every block drains one system at a time once
 * its team job (if any) is done.
 * Every system has its own convergence test, status and iteration count, and
 * runs exactly the iteration of hs_cg / hs_bicgstab (FP64).
 * A batch whose systems all name HS_SOLVER_MIXED runs FP64 iterative
 * refinement per system (the scheme of hs_solve_mixed) inside one kernel:
 * the FP64 residual b - A x is scaled by a power of two and rounded to FP32,
 * the correction equation is solved in FP32 (CG for symmetric operators,
 * BiCGStab for the upwind operator) to opts.inner_tol / opts.inner_maxit,
 * and x += correction in FP64, until the FP64 relative residual <= tol or
 * maxit refinement steps. */
typedef struct hs_batch hs_batch;   /* opaque, library-owned */

/* ops[s] (copied; a diffusion operator's k stays borrowed) and
 * solvers[s] in {HS_SOLVER_CG (symmetric operators), HS_SOLVER_BICGSTAB}, or
 * HS_SOLVER_MIXED for every system.  HS_ERR_INVALID for a NULL operator, an
 * unknown solver, CG on the upwind operator, or MIXED for only some systems. */
hs_status hs_batch_create(int nsys, const hs_op *const *ops, const int *solvers, hs_batch **out);
void hs_batch_destroy(hs_batch *batch);
/* Device workspace bytes for hs_batch_solve (plans the teams on first use). */
hs_status hs_batch_workspace_size(hs_batch *batch, size_t *bytes);
/* b[s], x[s]: host arrays of nsys FP64 device pointers (x: initial guess in,
 * solution out).  res: host array of nsys results (true_rel_res = -1 for FP64
 * systems; for mixed systems iters = outer = refinement steps, inner_iters =
 * their inner iterations, rel_res = true_rel_res = the FP64 relative residual,
 * restarts = inner BiCGStab restarts).
 * Returns HS_OK unless a system timed out or the launch failed; per-system
 * breakdowns and non-convergence are reported in res[s].status.  Calls on one
 * batch object are serialised by the library; the captured graph is reused
 * while ws and stream stay the same. */
hs_status hs_batch_solve(hs_batch *batch, const double *const *b, double *const *x, double tol,
                         int maxit, const hs_opts *opts, void *ws, size_t ws_bytes, void *stream,
                         hs_result *res);
/* Per-system z planes per work item (e.g. from the autotuner; 0 = cost
 * model).  planes: host array of nsys ints.  Re-plans the batch, so call it
 * before hs_batch_workspace_size. */
hs_status hs_batch_set_tile_planes(hs_batch *batch, const int *planes);
/* Introspection: 1 if the last solve replayed a CUDA graph; the grid size;
 * the team size (blocks) of every system. */
int hs_batch_graph_used(const hs_batch *batch);
int hs_batch_grid(const hs_batch *batch);
hs_status hs_batch_team_sizes(const hs_batch *batch, int *teams);

/* Diagnostics: runs one of the library's bounded device-side waits against a
 * condition that never comes true, to show that the wait gives up, reports
 * it and leaves the context usable.  kind:
 *   0  the grid reduce-barrier of the persistent solvers (a team of two
 *      blocks of which only one is launched),
 *   1  the Gauss-Seidel tile-dependency wait (a sweep count that nothing
 *      publishes),
 *   2  the 27-point Gauss-Seidel ring-neighbour wait (progress words that
 *      nothing publishes),
 *   3  the waits of the plane-lagged 27-point Gauss-Seidel (a block's wait for
 *      the plane above, its polling warp and the compute warps waiting on it,
 *      for plane counts that nothing publishes).
 * timeout_s: the wait's limit, 0 < timeout_s <= 10 seconds.  Allocates 4 KB of
 * device memory for the call and synchronises `stream`.
 * Returns HS_ERR_TIMEOUT when the wait gave up as designed, HS_OK if it ended
 * otherwise (a defect), HS_ERR_INVALID for a bad kind or limit, HS_ERR_CUDA
 * on a CUDA error. */
hs_status hs_diag_wait_timeout(int kind, double timeout_s, void *stream);

/* Diagnostics: the FP64 fused multiply-add rate of the current device in
 * flop/s (2 flops per FMA), measured on `stream` with independent FMA chains
 * in every resident thread (best of three timed launches of about 20 ms).
 * The FP64 solvers are bound by this rate; it is the roofline peak their
 * flop rates are quoted against.  Allocates 16 bytes of device memory for
 * the call and synchronises `stream`.  HS_ERR_INVALID for a NULL result
 * pointer, HS_ERR_CUDA on a CUDA error. */
hs_status hs_diag_fp64_rate(void *stream, double *flops_per_s);

/* Thread-local message describing the last non-OK status (never NULL). */
const char *hs_last_error(void);

/* 1 if the last hs_cg / hs_solve_mixed call on this thread ran its FP32
 * diffusion CG with TMA-staged planes (hs_opts.staging = 1), else 0. */
int hs_last_staging(void);

/* Library version string. */
const char *hs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HSOLVE_H */
