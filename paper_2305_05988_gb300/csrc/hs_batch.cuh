// hs_batch.cuh -- types shared by the two batched persistent kernels: the
// FP64 one (hs_batch.cu) and the mixed-precision one (hs_batch_mixed.cu),
// which is compiled on its own so both build in parallel.
#pragma once
#include "hs_krylov.cuh"

namespace hs {

struct BatchJob {
  int sys, rank, size, pad;
};

constexpr int BATCH_THREADS = 256;   // 8 rows per tile
// Minimum resident blocks per SM asked of the compiler for the batched
// kernels: four (64 registers) against its own choice of 128 (512-system
// batch, fresh tile tuning each run: FP64 16.8 -> 9.56 s, FP32-inner
// refinement 32.1 -> 9.38 s; three blocks: 9.70 / 9.68 s, two: 10.8 /
// 13.0 s).  More resident blocks give the large systems larger teams.
#ifndef HS_BATCH_MINBLOCKS
#define HS_BATCH_MINBLOCKS 4
#endif
#ifndef HS_BATCHMX_MINBLOCKS
#define HS_BATCHMX_MINBLOCKS 4
#endif
constexpr int BATCH_BY = BATCH_THREADS / 32;
// The batch kernels hold every iteration body at once, so they run them
// with one column per lane to keep their register count (and occupancy) down.
constexpr int BATCH_CX = 1;
// Per-system outcome written by the gather kernels: status, iterations (outer
// steps for mixed systems), relative residual, BiCGStab restarts, outer
// steps, inner iterations.
constexpr int BATCH_OUT = 6;

enum MxKind : int {
  MK_CG_SYM2 = 0,
  MK_CG_SYM3,
  MK_CG_VARK2,
  MK_CG_VARK3,
  MK_BI_SYM2,
  MK_BI_SYM3,
  MK_BI_NONSYM2,
  MK_BI_NONSYM3,
  MK_BI_VARK2,
  MK_BI_VARK3,
};

// One system of a mixed-precision batch: FP64 iterative refinement whose
// correction equation is solved by FP32 CG (symmetric operators) or FP32
// BiCGStab (the upwind operator), as in hs_solve_mixed.
struct MxSys {
  int kind;              // MxKind
  int max_outer;         // refinement steps
  double tol;            // FP64 relative residual
  double restart_eps;    // inner BiCGStab restart threshold for a unit-norm right-hand side
  double inner_tol;      // inner relative tolerance (tightest)
  int inner_fixed;       // 1: every inner solve to inner_tol; 0: a step near tol stops earlier
  int pad_;
  Geom g;
  Tiling tl;             // tiling of the FP64 residual pass
  Coef<double> cf;       // FP64 operator (scaled form, A = sigma * cf)
  double sigma;
  const double* b;
  double* x;
  float* r32;            // scaled residual, right-hand side of the inner solve
  float* d32;            // inner solution (scaled correction)
  Common cm;             // outer control block; partials shared with the inner solve
  Ctrl* inner_ctrl;
  CgArgs<float> cg;      // inner CG: b = r32, x = d32
  BiArgs<float> bi;      // inner BiCGStab: b = r32, x = d32
};
static_assert(sizeof(MxSys) % 8 == 0, "descriptor must be copied in 8-byte words");

// Host entry points of the mixed-precision batch kernel (hs_batch_mixed.cu).
int batch_mx_blocks_per_sm(int threads, size_t smem);
cudaError_t batch_mx_launch(cudaStream_t s, int grid, size_t smem, const MxSys* sys, int nsys,
                            unsigned long long timeout_ns, const int* job_off, const BatchJob* jobs, const int* queue,
                            int nqueue, int* head, double* out);

}  // namespace hs
