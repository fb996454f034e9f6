/*
 * oracle.c -- plain, slow, sequential FP64 CPU oracle for the structured-grid
 * iterative solvers of Martinez-Ferrer, Arslan & Beltran, "Improving the
 * performance of classical linear algebra iterative methods via hybrid
 * parallelism" (arXiv 2305.05988).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check of the
 * package entry module and the CPU-baseline leg of the benchmark may load
 * this library.  It shares no code, header, table or helper with the CUDA
 * path and never calls it.
 *
 * Every loop runs in lexicographic order idx = i + nx*(j + ny*k) (i fastest),
 * every stencil sum is a plain left-to-right sum, inner products are the
 * exact sum of the rounded products to within a few units in the last place
 * (compensated summation, see ora_dot), and the file is compiled with
 * -O2 -ffp-contract=off so that no fused multiply-add reorders the rounding.
 *
 * Operators (readings of points the paper leaves open; the paper solves
 * A x = b with a sparse A arising from a centred-stencil PDE discretisation,
 * section 3.1 and section 4.1):
 *   - grid of interior nodes n_d per dimension, h_d = 1/(n_d + 1),
 *     homogeneous Dirichlet boundary (ghost value 0);
 *   - LAPLACIAN  A = -Delta_h: diagonal sum_d 2/h_d^2, neighbours -1/h_d^2;
 *   - UPWIND     -Delta u + beta . grad u, beta_d >= 0, first-order upwind:
 *                diagonal sum_d (2/h_d^2 + beta_d/h_d), lower neighbour
 *                -1/h_d^2 - beta_d/h_d, upper neighbour -1/h_d^2;
 *   - DIFFUSION  -div(k grad u), face coefficient kappa = 2 k_i k_j/(k_i+k_j)
 *                (harmonic mean), a boundary face uses kappa = k_i; diagonal
 *                sum_f kappa_f/h_d^2, neighbour -kappa_f/h_d^2;
 *   - HPCG7 / HPCG27  the benchmark system of section 4.1 (HPCG's generated
 *                matrix, unscaled): diagonal 27, -1 for each of the 6 face
 *                neighbours (7-point) or all 26 neighbours (27-point) inside
 *                the grid.  The paper does not print the coefficients; 27 on
 *                the diagonal with both stencils is the reading that fits its
 *                printed iteration counts (a diagonal of 26 or 6 would make
 *                Jacobi stall far above eps = 1e-6), see the golden counts.
 *
 * Parity status of each function is stated beside it; all are pinned by the
 * CPU tests (dense assembly, closed-form eigenpairs, dense LU solves, dense
 * triangular solves, finite termination, finite differences).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

/*
 * Element-wise loops (every iteration writes its own entries and reads only
 * data no iteration writes) may run on several threads when this file is
 * compiled with OpenMP: the result is bitwise that of the sequential loop.
 * Inner products, the Gauss-Seidel sweeps and everything else stay
 * sequential.  The parity checker is built without OpenMP.
 */
#ifdef _OPENMP
#include <omp.h>
#define ORA_PARALLEL_FOR _Pragma("omp parallel for schedule(static)")
#else
#define ORA_PARALLEL_FOR
#endif

void ora_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int ora_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Operator rows                                                            */
/* ------------------------------------------------------------------------ */

static double harmonic(double a, double b) { return 2.0 * a * b / (a + b); }

static double dharmonic_da(double a, double b)
{
    /* d/da [2ab/(a+b)] = 2 b^2 / (a+b)^2 */
    double s = a + b;
    return 2.0 * b * b / (s * s);
}

/* Coordinates of a lexicographic index. */
static void coords(const ora_op *A, int64_t idx, int64_t c[3])
{
    c[0] = idx % A->n[0];
    c[1] = (idx / A->n[0]) % A->n[1];
    c[2] = idx / (A->n[0] * A->n[1]);
}

static int64_t stride_of(const ora_op *A, int d)
{
    if (d == 0) return 1;
    if (d == 1) return A->n[0];
    return A->n[0] * A->n[1];
}

int64_t ora_size(const ora_op *A)
{
    int64_t N = 1;
    for (int d = 0; d < A->ndim; d++) N *= A->n[d];
    return N;
}

/*
 * Row `idx` of the operator: its diagonal and its off-diagonal entries.
 * Off-diagonal neighbours outside the grid are dropped (zero ghost value).
 * Entries are listed dimension by dimension, lower neighbour before upper.
 * Returns the number of off-diagonal entries written to nb[] / c[].
 */
int ora_row(const ora_op *A, int64_t idx, double *diag, int64_t nb[ORA_MAXNB], double c[ORA_MAXNB])
{
    int64_t x[3] = {0, 0, 0};
    coords(A, idx, x);
    int cnt = 0;
    double dg = 0.0;
    if (A->kind == ORA_HPCG27) {
        /* all neighbours of the 3x3x3 box, in lexicographic order */
        for (int dz = -1; dz <= 1; dz++)
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    if (dx == 0 && dy == 0 && dz == 0) continue;
                    int64_t xi = x[0] + dx, yj = x[1] + dy, zk = x[2] + dz;
                    if (xi < 0 || xi >= A->n[0] || yj < 0 || yj >= A->n[1] || zk < 0 || zk >= A->n[2])
                        continue;
                    nb[cnt] = xi + A->n[0] * (yj + A->n[1] * zk);
                    c[cnt] = -1.0;
                    cnt++;
                }
        *diag = 27.0;
        return cnt;
    }
    if (A->kind == ORA_HPCG7) {
        for (int d = 0; d < A->ndim; d++) {
            int64_t s = stride_of(A, d);
            if (x[d] > 0)            { nb[cnt] = idx - s; c[cnt] = -1.0; cnt++; }
            if (x[d] < A->n[d] - 1)  { nb[cnt] = idx + s; c[cnt] = -1.0; cnt++; }
        }
        *diag = 27.0;
        return cnt;
    }
    for (int d = 0; d < A->ndim; d++) {
        double ih2 = 1.0 / (A->h[d] * A->h[d]);
        int64_t s = stride_of(A, d);
        for (int side = 0; side < 2; side++) {      /* 0 = lower, 1 = upper */
            int inside = side == 0 ? (x[d] > 0) : (x[d] < A->n[d] - 1);
            int64_t j = side == 0 ? idx - s : idx + s;
            double off;                              /* off-diagonal entry */
            double dpart;                            /* diagonal contribution */
            if (A->kind == ORA_LAPLACIAN) {
                off = -ih2;
                dpart = ih2;
            } else if (A->kind == ORA_UPWIND) {
                double bh = A->beta[d] / A->h[d];
                if (side == 0) { off = -ih2 - bh; dpart = ih2 + bh; }
                else           { off = -ih2;      dpart = ih2; }
            } else {
                double kap = inside ? harmonic(A->k[idx], A->k[j]) : A->k[idx];
                off = -kap * ih2;
                dpart = kap * ih2;
            }
            dg += dpart;
            if (inside) { nb[cnt] = j; c[cnt] = off; cnt++; }
        }
    }
    *diag = dg;
    return cnt;
}

/* y = A x, row by row (the sparse matrix-vector product, section 3.1). */
void ora_spmv(const ora_op *A, const double *x, double *y)
{
    int64_t N = ora_size(A);
    ORA_PARALLEL_FOR
    for (int64_t i = 0; i < N; i++) {
        double dg, c[ORA_MAXNB];
        int64_t nb[ORA_MAXNB];
        int m = ora_row(A, i, &dg, nb, c);
        double acc = dg * x[i];
        for (int q = 0; q < m; q++) acc += c[q] * x[nb[q]];
        y[i] = acc;
    }
}

/* Dense row-major N x N copy of the operator (tiny grids only). */
int ora_dense(const ora_op *A, double *M, int64_t maxN)
{
    int64_t N = ora_size(A);
    if (N > maxN) return -1;
    memset(M, 0, (size_t)(N * N) * sizeof(double));
    for (int64_t i = 0; i < N; i++) {
        double dg, c[ORA_MAXNB];
        int64_t nb[ORA_MAXNB];
        int m = ora_row(A, i, &dg, nb, c);
        M[i * N + i] = dg;
        for (int q = 0; q < m; q++) M[i * N + nb[q]] += c[q];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Vector helpers (plain sequential loops)                                  */
/* ------------------------------------------------------------------------ */

/*
 * Inner product sum_i a_i b_i.  The terms are added in index order with
 * Neumaier's compensated summation (A. Neumaier, "Rundungsfehleranalyse
 * einiger Verfahren zur Summation endlicher Summen", ZAMM 54, 1974): the
 * rounding error of every addition is carried in c and added back at the
 * end, so the result stays within a few units of the exactly rounded sum of
 * the rounded products instead of drifting by O(N) units with the length.
 */
double ora_dot(int64_t N, const double *a, const double *b)
{
    double s = 0.0, c = 0.0;
    for (int64_t i = 0; i < N; i++) {
        double t = a[i] * b[i];
        double u = s + t;
        if (fabs(s) >= fabs(t)) c += (s - u) + t;
        else                    c += (t - u) + s;
        s = u;
    }
    return s + c;
}

/* r = b - A x */
void ora_residual(const ora_op *A, const double *b, const double *x, double *r)
{
    int64_t N = ora_size(A);
    ora_spmv(A, x, r);
    ORA_PARALLEL_FOR
    for (int64_t i = 0; i < N; i++) r[i] = b[i] - r[i];
}

/* ||b - A x||_2 / ||b||_2 (0 when b = 0 and x = 0). */
double ora_relres(const ora_op *A, const double *b, const double *x)
{
    int64_t N = ora_size(A);
    double *r = (double *)malloc((size_t)N * sizeof(double));
    if (!r) return NAN;
    ora_residual(A, b, x, r);
    double rn = sqrt(ora_dot(N, r, r));
    double bn = sqrt(ora_dot(N, b, b));
    free(r);
    if (bn == 0.0) return rn == 0.0 ? 0.0 : INFINITY;
    return rn / bn;
}

/* ------------------------------------------------------------------------ */
/* Jacobi (section 3.1): x_i <- (b_i - sum_{j != i} a_ij x_j) / a_ii,       */
/* undamped, every update reading the previous iterate only.                */
/* ------------------------------------------------------------------------ */

/*
 * Runs up to `maxit` sweeps.  With tol > 0 the relative residual of the
 * current iterate is tested before each sweep and the loop returns the first
 * iterate x_k with ||b - A x_k|| / ||b|| <= tol (iteration count k).  With
 * tol == 0 exactly `maxit` sweeps run.  hist (may be NULL) receives the
 * relative residual of x_0 .. x_k when tol > 0.
 */
int ora_jacobi(const ora_op *A, const double *b, double *x, int maxit, double tol,
               double *hist, int *iters)
{
    int64_t N = ora_size(A);
    double *xn = (double *)malloc((size_t)N * sizeof(double));
    if (!xn) return -1;
    double bn = sqrt(ora_dot(N, b, b));
    int status = ORA_NOT_CONVERGED;
    int k = 0;
    for (k = 0;; k++) {
        if (tol > 0.0) {
            double rr = ora_relres(A, b, x);
            if (bn == 0.0) rr = 0.0;
            if (hist) hist[k] = rr;
            if (rr <= tol) { status = ORA_OK; break; }
        }
        if (k == maxit) break;
        ORA_PARALLEL_FOR
        for (int64_t i = 0; i < N; i++) {
            double dg, c[ORA_MAXNB];
            int64_t nb[ORA_MAXNB];
            int m = ora_row(A, i, &dg, nb, c);
            double acc = b[i];
            for (int q = 0; q < m; q++) acc -= c[q] * x[nb[q]];
            xn[i] = acc / dg;
        }
        memcpy(x, xn, (size_t)N * sizeof(double));
    }
    if (tol == 0.0) status = ORA_OK;
    free(xn);
    *iters = k;
    return status;
}

/* ------------------------------------------------------------------------ */
/* Gauss-Seidel (section 3.1): in-place sweeps that use every entry already */
/* updated in the current sweep.  Forward visits idx ascending, backward    */
/* descending; the symmetric method is one forward then one backward sweep  */
/* per iteration.                                                           */
/* ------------------------------------------------------------------------ */

static void gs_point(const ora_op *A, const double *b, double *x, int64_t i)
{
    double dg, c[ORA_MAXNB];
    int64_t nb[ORA_MAXNB];
    int m = ora_row(A, i, &dg, nb, c);
    double acc = b[i];
    for (int q = 0; q < m; q++) acc -= c[q] * x[nb[q]];
    x[i] = acc / dg;
}

void ora_gs_sweep(const ora_op *A, const double *b, double *x, int backward)
{
    int64_t N = ora_size(A);
    if (!backward)
        for (int64_t i = 0; i < N; i++) gs_point(A, b, x, i);
    else
        for (int64_t i = N - 1; i >= 0; i--) gs_point(A, b, x, i);
}

/*
 * mode: ORA_GS_FORWARD / ORA_GS_BACKWARD (one sweep per iteration) or
 * ORA_GS_SYMMETRIC (forward + backward per iteration).  Stopping rule and
 * history as in ora_jacobi.
 */
int ora_gauss_seidel(const ora_op *A, const double *b, double *x, int maxit, double tol,
                     int mode, double *hist, int *iters)
{
    int64_t N = ora_size(A);
    double bn = sqrt(ora_dot(N, b, b));
    int status = ORA_NOT_CONVERGED;
    int k;
    for (k = 0;; k++) {
        if (tol > 0.0) {
            double rr = ora_relres(A, b, x);
            if (bn == 0.0) rr = 0.0;
            if (hist) hist[k] = rr;
            if (rr <= tol) { status = ORA_OK; break; }
        }
        if (k == maxit) break;
        if (mode == ORA_GS_FORWARD || mode == ORA_GS_SYMMETRIC) ora_gs_sweep(A, b, x, 0);
        if (mode == ORA_GS_BACKWARD || mode == ORA_GS_SYMMETRIC) ora_gs_sweep(A, b, x, 1);
    }
    if (tol == 0.0) status = ORA_OK;
    *iters = k;
    return status;
}

/* ------------------------------------------------------------------------ */
/* Conjugate gradient: the classical Hestenes-Stiefel iteration that HPCCG  */
/* runs (section 3.2), stopped on the recursive relative residual.          */
/* ------------------------------------------------------------------------ */

int ora_cg(const ora_op *A, const double *b, double *x, int maxit, double tol,
           double *hist, int *iters)
{
    int64_t N = ora_size(A);
    double *r = (double *)malloc((size_t)N * sizeof(double));
    double *p = (double *)malloc((size_t)N * sizeof(double));
    double *w = (double *)malloc((size_t)N * sizeof(double));
    if (!r || !p || !w) { free(r); free(p); free(w); return -1; }
    int status = ORA_NOT_CONVERGED;
    int it = 0;
    double bn = sqrt(ora_dot(N, b, b));
    if (bn == 0.0) {
        ORA_PARALLEL_FOR
        for (int64_t i = 0; i < N; i++) x[i] = 0.0;
        if (hist) hist[0] = 0.0;
        *iters = 0;
        free(r); free(p); free(w);
        return ORA_OK;
    }
    ora_residual(A, b, x, r);
    ORA_PARALLEL_FOR
    for (int64_t i = 0; i < N; i++) p[i] = r[i];
    double rr = ora_dot(N, r, r);
    if (hist) hist[0] = sqrt(rr) / bn;
    if (sqrt(rr) / bn <= tol) status = ORA_OK;
    while (status != ORA_OK && it < maxit) {
        ora_spmv(A, p, w);
        double pw = ora_dot(N, p, w);
        if (!(pw > 0.0)) { status = ORA_BREAKDOWN; break; }
        double alpha = rr / pw;
        ORA_PARALLEL_FOR
        for (int64_t i = 0; i < N; i++) x[i] += alpha * p[i];
        ORA_PARALLEL_FOR
        for (int64_t i = 0; i < N; i++) r[i] -= alpha * w[i];
        double rr_new = ora_dot(N, r, r);
        it++;
        if (hist) hist[it] = sqrt(rr_new) / bn;
        if (sqrt(rr_new) / bn <= tol) { status = ORA_OK; break; }
        double beta = rr_new / rr;
        ORA_PARALLEL_FOR
        for (int64_t i = 0; i < N; i++) p[i] = r[i] + beta * p[i];
        rr = rr_new;
    }
    *iters = it;
    free(r); free(p); free(w);
    return status;
}

/* ------------------------------------------------------------------------ */
/* BiCGStab with the normalised shadow residual and the restart rule of     */
/* Algorithm 2 (r' = r0/||r0||, restart when sqrt|alpha_n| < eps'), in the  */
/* classical statement order: the convergence test follows each residual    */
/* update and the converged iterate is returned.                            */
/* ------------------------------------------------------------------------ */

int ora_bicgstab(const ora_op *A, const double *b, double *x, int maxit, double tol,
                 double restart_eps, double *hist, int *iters, int *restarts,
                 double *trace, int *restart_at)
{
    int64_t N = ora_size(A);
    double *r = (double *)malloc((size_t)N * sizeof(double));
    double *rs = (double *)malloc((size_t)N * sizeof(double));  /* r'   */
    double *p = (double *)malloc((size_t)N * sizeof(double));
    double *v = (double *)malloc((size_t)N * sizeof(double));   /* A p  */
    double *s = (double *)malloc((size_t)N * sizeof(double));
    double *t = (double *)malloc((size_t)N * sizeof(double));   /* A s  */
    int status = ORA_NOT_CONVERGED;
    int it = 0, nrestart = 0;
    if (!r || !rs || !p || !v || !s || !t) { status = -1; goto done; }
    double bn = sqrt(ora_dot(N, b, b));
    if (bn == 0.0) {
        ORA_PARALLEL_FOR
        for (int64_t i = 0; i < N; i++) x[i] = 0.0;
        if (hist) hist[0] = 0.0;
        status = ORA_OK;
        goto done;
    }
    ora_residual(A, b, x, r);
    double beta_r = ora_dot(N, r, r);
    if (hist) hist[0] = sqrt(beta_r) / bn;
    if (sqrt(beta_r) / bn <= tol) { status = ORA_OK; goto done; }
    double rn = sqrt(beta_r);
    ORA_PARALLEL_FOR
    for (int64_t i = 0; i < N; i++) rs[i] = r[i] / rn;
    double alpha_n = ora_dot(N, r, rs);
    if (trace) trace[0] = alpha_n;
    ORA_PARALLEL_FOR
    for (int64_t i = 0; i < N; i++) p[i] = r[i];
    while (it < maxit) {
        ora_spmv(A, p, v);
        double alpha_d = ora_dot(N, v, rs);
        if (alpha_d == 0.0 || !isfinite(alpha_d)) { status = ORA_BREAKDOWN; break; }
        double alpha = alpha_n / alpha_d;
        ORA_PARALLEL_FOR
        for (int64_t i = 0; i < N; i++) s[i] = r[i] - alpha * v[i];
        double ss = ora_dot(N, s, s);
        it++;
        if (sqrt(ss) / bn <= tol) {
            ORA_PARALLEL_FOR
            for (int64_t i = 0; i < N; i++) x[i] += alpha * p[i];
            if (hist) hist[it] = sqrt(ss) / bn;
            status = ORA_OK;
            break;
        }
        ora_spmv(A, s, t);
        double ts = ora_dot(N, t, s);
        double tt = ora_dot(N, t, t);
        if (tt == 0.0 || !isfinite(tt)) { status = ORA_BREAKDOWN; break; }
        double omega = ts / tt;
        if (omega == 0.0) { status = ORA_BREAKDOWN; break; }
        ORA_PARALLEL_FOR
        for (int64_t i = 0; i < N; i++) x[i] += alpha * p[i] + omega * s[i];
        ORA_PARALLEL_FOR
        for (int64_t i = 0; i < N; i++) r[i] = s[i] - omega * t[i];
        double alpha_n_new = ora_dot(N, r, rs);
        beta_r = ora_dot(N, r, r);
        if (hist) hist[it] = sqrt(beta_r) / bn;
        if (trace) trace[it] = alpha_n_new;      /* the value the restart test reads */
        if (sqrt(beta_r) / bn <= tol) { status = ORA_OK; break; }
        if (restart_eps > 0.0 && sqrt(fabs(alpha_n_new)) < restart_eps) {
            /* restart: new search direction and new shadow residual */
            double rnorm = sqrt(beta_r);
            ORA_PARALLEL_FOR
            for (int64_t i = 0; i < N; i++) p[i] = r[i];
            ORA_PARALLEL_FOR
            for (int64_t i = 0; i < N; i++) rs[i] = r[i] / rnorm;
            alpha_n = ora_dot(N, r, rs);
            if (restart_at) restart_at[nrestart] = it;
            nrestart++;
        } else {
            double beta = alpha_n_new / (alpha_d * omega);
            ORA_PARALLEL_FOR
            for (int64_t i = 0; i < N; i++) p[i] = r[i] + beta * (p[i] - omega * v[i]);
            alpha_n = alpha_n_new;
        }
    }
done:
    *iters = it;
    if (restarts) *restarts = nrestart;
    free(r); free(rs); free(p); free(v); free(s); free(t);
    return status;
}

/* ------------------------------------------------------------------------ */
/* CG-NB, the paper's nonblocking CG (section 3.2, Algorithm 1): the SpMV is */
/* applied to r_j and A p_j follows from the recurrence                     */
/*   A p_j = A r_j + (alpha_n,j / alpha_n,j-1) A p_j-1,                      */
/* the search direction p_j = r_j + (alpha_n,j / alpha_n,j-1) p_j-1 and      */
/*   x_j = x_j-1 + alpha_n,j-1^2 / (alpha_d,j-1 alpha_n,j) (p_j - r_j),      */
/* with alpha_n = r.r, alpha_d = (A p).p.  The printed x update carries a    */
/* minus sign; with r_j = r_j-1 - alpha_j-1 A p_j-1 the derivation gives     */
/* plus (p_j - r_j = beta_j p_j-1), the reading used here.                   */
/* Stopping: relative residual sqrt(alpha_n,j)/||b|| <= tol tested at the     */
/* end of iteration j, returning x_j (iters = j).  paper_order = 1 tests at  */
/* the top of the next iteration instead and applies the printed final      */
/* step x = x_l + alpha_l p_l after the loop.                               */
/* ------------------------------------------------------------------------ */

int ora_cg_nb(const ora_op *A, const double *b, double *x, int maxit, double tol,
              int paper_order, double *hist, int *iters)
{
    int64_t N = ora_size(A);
    double *r = (double *)malloc((size_t)N * sizeof(double));
    double *p = (double *)malloc((size_t)N * sizeof(double));
    double *Ap = (double *)malloc((size_t)N * sizeof(double));
    double *Ar = (double *)malloc((size_t)N * sizeof(double));
    int status = ORA_NOT_CONVERGED, it = 0;
    if (!r || !p || !Ap || !Ar) { status = -1; goto done; }
    double bn = sqrt(ora_dot(N, b, b));
    if (bn == 0.0) {
        ORA_PARALLEL_FOR
        for (int64_t i = 0; i < N; i++) x[i] = 0.0;
        if (hist) hist[0] = 0.0;
        status = ORA_OK;
        goto done;
    }
    /* r0 = b - A x0, p0 = r0, alpha_0 = (r0.r0) / ((A p0).p0) */
    ora_residual(A, b, x, r);
    ORA_PARALLEL_FOR
    for (int64_t i = 0; i < N; i++) p[i] = r[i];
    ora_spmv(A, p, Ap);
    double an = ora_dot(N, r, r);
    double ad = ora_dot(N, Ap, p);
    if (hist) hist[0] = sqrt(an) / bn;
    if (sqrt(an) / bn <= tol) { status = ORA_OK; goto done; }
    if (!(ad > 0.0)) { status = ORA_BREAKDOWN; goto done; }
    double alpha = an / ad;
    for (it = 1; it <= maxit; it++) {
        if (paper_order && sqrt(an) / bn <= tol && it > 1) { it--; status = ORA_OK; break; }
        ORA_PARALLEL_FOR
        for (int64_t i = 0; i < N; i++) r[i] -= alpha * Ap[i];
        double an_new = ora_dot(N, r, r);
        double beta = an_new / an;
        ora_spmv(A, r, Ar);
        ORA_PARALLEL_FOR
        for (int64_t i = 0; i < N; i++) Ap[i] = Ar[i] + beta * Ap[i];
        ORA_PARALLEL_FOR
        for (int64_t i = 0; i < N; i++) p[i] = r[i] + beta * p[i];
        double ad_new = ora_dot(N, Ap, p);
        double c = an * an / (ad * an_new);
        ORA_PARALLEL_FOR
        for (int64_t i = 0; i < N; i++) x[i] += c * (p[i] - r[i]);
        if (hist) hist[it] = sqrt(an_new) / bn;
        an = an_new;
        ad = ad_new;
        if (!paper_order && sqrt(an) / bn <= tol) { status = ORA_OK; break; }
        if (!(ad > 0.0)) { status = ORA_BREAKDOWN; break; }
        alpha = an / ad;
    }
    if (it > maxit) it = maxit;
    if (paper_order && status != ORA_BREAKDOWN) {
        /* the printed final step x = x_l + alpha_l p_l */
        ORA_PARALLEL_FOR
        for (int64_t i = 0; i < N; i++) x[i] += alpha * p[i];
        if (status != ORA_OK && sqrt(an) / bn <= tol) status = ORA_OK;
    }
done:
    *iters = it;
    free(r); free(p); free(Ap); free(Ar);
    return status;
}

/* ------------------------------------------------------------------------ */
/* BiCGStab-B1, the statement order of Algorithm 2 (section 3.2): in        */
/* iteration j the convergence test on beta_j = r_j.r_j comes after         */
/* alpha_d,j, s_j, omega_j and x_j+1/2 = x_j + alpha_j p_j, and the loop     */
/* ends with the printed final step x = x_l + omega_l s_l, so the returned   */
/* iterate is x_l+1 for the first l with sqrt(beta_l)/||b|| <= tol           */
/* (iters = l + 1 SpMV pairs).  Restart as in ora_bicgstab.                 */
/* ------------------------------------------------------------------------ */

int ora_bicgstab_b1(const ora_op *A, const double *b, double *x, int maxit, double tol,
                    double restart_eps, double *hist, int *iters, int *restarts)
{
    int64_t N = ora_size(A);
    double *r = (double *)malloc((size_t)N * sizeof(double));
    double *rs = (double *)malloc((size_t)N * sizeof(double));
    double *p = (double *)malloc((size_t)N * sizeof(double));
    double *Ap = (double *)malloc((size_t)N * sizeof(double));
    double *s = (double *)malloc((size_t)N * sizeof(double));
    double *As = (double *)malloc((size_t)N * sizeof(double));
    int status = ORA_NOT_CONVERGED, it = 0, nrestart = 0;
    if (!r || !rs || !p || !Ap || !s || !As) { status = -1; goto done; }
    double bn = sqrt(ora_dot(N, b, b));
    if (bn == 0.0) {
        ORA_PARALLEL_FOR
        for (int64_t i = 0; i < N; i++) x[i] = 0.0;
        if (hist) hist[0] = 0.0;
        status = ORA_OK;
        goto done;
    }
    ora_residual(A, b, x, r);
    double beta_j = ora_dot(N, r, r);
    if (hist) hist[0] = sqrt(beta_j) / bn;
    if (sqrt(beta_j) / bn <= tol) { status = ORA_OK; goto done; }
    ORA_PARALLEL_FOR
    for (int64_t i = 0; i < N; i++) rs[i] = r[i] / sqrt(beta_j);
    double an = ora_dot(N, r, rs);
    ORA_PARALLEL_FOR
    for (int64_t i = 0; i < N; i++) p[i] = r[i];
    while (it < maxit) {
        ora_spmv(A, p, Ap);
        double ad = ora_dot(N, Ap, rs);
        if (ad == 0.0 || !isfinite(ad)) { status = ORA_BREAKDOWN; break; }
        double alpha = an / ad;
        ORA_PARALLEL_FOR
        for (int64_t i = 0; i < N; i++) s[i] = r[i] - alpha * Ap[i];
        ora_spmv(A, s, As);
        double num = ora_dot(N, As, s), den = ora_dot(N, As, As);
        if (den == 0.0 || !isfinite(den)) { status = ORA_BREAKDOWN; break; }
        double omega = num / den;
        ORA_PARALLEL_FOR
        for (int64_t i = 0; i < N; i++) x[i] += alpha * p[i];            /* x_j+1/2 */
        it++;
        if (sqrt(beta_j) / bn <= tol) {                                  /* late test */
            ORA_PARALLEL_FOR
            for (int64_t i = 0; i < N; i++) x[i] += omega * s[i];        /* final step */
            status = ORA_OK;
            break;
        }
        ORA_PARALLEL_FOR
        for (int64_t i = 0; i < N; i++) x[i] += omega * s[i];
        ORA_PARALLEL_FOR
        for (int64_t i = 0; i < N; i++) r[i] = s[i] - omega * As[i];
        double an_new = ora_dot(N, r, rs);
        beta_j = ora_dot(N, r, r);
        if (hist) hist[it] = sqrt(beta_j) / bn;
        ORA_PARALLEL_FOR
        for (int64_t i = 0; i < N; i++) Ap[i] = p[i] - omega * Ap[i];   /* p_j+1/2, stored in Ap */
        if (restart_eps > 0.0 && sqrt(fabs(an_new)) < restart_eps) {
            ORA_PARALLEL_FOR
            for (int64_t i = 0; i < N; i++) p[i] = r[i];
            ORA_PARALLEL_FOR
            for (int64_t i = 0; i < N; i++) rs[i] = r[i] / sqrt(beta_j);
            an = ora_dot(N, r, rs);
            nrestart++;
        } else {
            double c = an_new / (ad * omega);
            ORA_PARALLEL_FOR
            for (int64_t i = 0; i < N; i++) p[i] = r[i] + c * Ap[i];
            an = an_new;
        }
    }
done:
    *iters = it;
    if (restarts) *restarts = nrestart;
    free(r); free(rs); free(p); free(Ap); free(s); free(As);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Adjoint gradient of L(u) for the diffusion operator.                     */
/* With A(k) u = f and lambda solving A^T lambda = dL/du:                   */
/*   dL/dk_i = -lambda^T (dA/dk_i) u                                        */
/*           = -sum_{faces f of cell i} dkappa_f/dk_i                       */
/*                 (lambda_i - lambda_j)(u_i - u_j) / h_d^2,                */
/* a boundary face contributing dkappa/dk_i = 1 with lambda_j = u_j = 0.    */
/* The output is g_i = dL/dlog k_i = k_i dL/dk_i.                           */
/* ------------------------------------------------------------------------ */

int ora_grad_logk(const ora_op *A, const double *u, const double *lam, double *g)
{
    if (A->kind != ORA_DIFFUSION) return -1;
    int64_t N = ora_size(A);
    ORA_PARALLEL_FOR
    for (int64_t i = 0; i < N; i++) {
        int64_t x[3] = {0, 0, 0};
        coords(A, i, x);
        double acc = 0.0;
        for (int d = 0; d < A->ndim; d++) {
            double ih2 = 1.0 / (A->h[d] * A->h[d]);
            int64_t s = stride_of(A, d);
            for (int side = 0; side < 2; side++) {
                int inside = side == 0 ? (x[d] > 0) : (x[d] < A->n[d] - 1);
                if (inside) {
                    int64_t j = side == 0 ? i - s : i + s;
                    double dk = dharmonic_da(A->k[i], A->k[j]);
                    acc += dk * (lam[i] - lam[j]) * (u[i] - u[j]) * ih2;
                } else {
                    acc += lam[i] * u[i] * ih2;
                }
            }
        }
        g[i] = -A->k[i] * acc;
    }
    return 0;
}
