/*
 * oracle.h -- declarations of the FP64 CPU oracle (test infrastructure only;
 * see oracle.c).  This header belongs to the oracle alone: the CUDA library
 * has its own, unrelated header.
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stdint.h>

enum { ORA_LAPLACIAN = 0, ORA_UPWIND = 1, ORA_DIFFUSION = 2, ORA_HPCG7 = 3, ORA_HPCG27 = 4 };
enum { ORA_MAXNB = 26 };   /* off-diagonal entries per row, at most */
enum { ORA_GS_FORWARD = 0, ORA_GS_BACKWARD = 1, ORA_GS_SYMMETRIC = 2 };
enum { ORA_OK = 0, ORA_NOT_CONVERGED = 1, ORA_BREAKDOWN = -3 };

typedef struct {
    int ndim;           /* 2 or 3 (1 allowed for tests)                 */
    int kind;           /* ORA_LAPLACIAN / ORA_UPWIND / ORA_DIFFUSION / ORA_HPCG7 / ORA_HPCG27 */
    int64_t n[3];       /* interior nodes per dimension (unused = 1)    */
    double h[3];        /* mesh spacing 1/(n_d + 1)                     */
    double beta[3];     /* upwind velocity, beta_d >= 0                 */
    const double *k;    /* per-cell diffusion coefficient (borrowed)    */
} ora_op;

int64_t ora_size(const ora_op *A);
int ora_row(const ora_op *A, int64_t idx, double *diag, int64_t nb[ORA_MAXNB], double c[ORA_MAXNB]);
void ora_spmv(const ora_op *A, const double *x, double *y);
int ora_dense(const ora_op *A, double *M, int64_t maxN);
double ora_dot(int64_t N, const double *a, const double *b);
void ora_residual(const ora_op *A, const double *b, const double *x, double *r);
double ora_relres(const ora_op *A, const double *b, const double *x);
int ora_jacobi(const ora_op *A, const double *b, double *x, int maxit, double tol,
               double *hist, int *iters);
void ora_gs_sweep(const ora_op *A, const double *b, double *x, int backward);
int ora_gauss_seidel(const ora_op *A, const double *b, double *x, int maxit, double tol,
                     int mode, double *hist, int *iters);
int ora_cg(const ora_op *A, const double *b, double *x, int maxit, double tol,
           double *hist, int *iters);
/* trace (may be NULL, maxit + 1 entries): trace[k] = r_k . r', the value the
 * restart test reads after iteration k (trace[0] = r_0 . r').  restart_at (may
 * be NULL, maxit entries): the iterations after which a restart was taken. */
int ora_bicgstab(const ora_op *A, const double *b, double *x, int maxit, double tol,
                 double restart_eps, double *hist, int *iters, int *restarts,
                 double *trace, int *restart_at);
int ora_cg_nb(const ora_op *A, const double *b, double *x, int maxit, double tol,
              int paper_order, double *hist, int *iters);
int ora_bicgstab_b1(const ora_op *A, const double *b, double *x, int maxit, double tol,
                    double restart_eps, double *hist, int *iters, int *restarts);
int ora_grad_logk(const ora_op *A, const double *u, const double *lam, double *g);
/* Threads of the element-wise loops (OpenMP build only; 1 otherwise). */
void ora_set_threads(int n);
int ora_threads(void);

#endif
