// hs_gs.cuh -- pieces shared by the three schedules of exactly lexicographic
// Gauss-Seidel (section 3.1): the kernel arguments, the two-part node update
// every schedule applies (gs_old, then gs_new), the grid residual, the
// bounded progress wait, and the host set-up and finish of a solve.
//
// The schedules:
//   * hs_gs.cu   -- the dataflow tile schedule (k_gs, any 2-/3-D grid), the
//                   workspace sizing and the dispatch between schedules;
//   * hs_gsp.cu  -- the pencil schedule (k_gsp, pipelined batches on 3-D
//                   constant-coefficient operators);
//   * hs_gs2d.cu -- small 1-/2-D grids held on chip by one block (k_gs2d) or
//                   by one thread-block cluster (k_gs2dc).
// All of them reproduce the sequential sweep up to the rounding order inside
// a single update, and give bitwise the same iterates as each other.
#pragma once
#include <math.h>

#include <algorithm>

#include "hs_internal.h"

namespace hs {

template <typename T>
struct GsArgs {
  Geom g;
  Coef<T> cf;           // Jacobi-form couplings (g = -a/a_ii) or var-k arrays (D = 1/a_ii)
  T invd;
  double dscale2;
  const T* b;
  T* bD;
  T* x;
  Common cm;
  const int* plane_off;   // P + 1 offsets into plane_tiles
  const int* plane_tiles; // tile ids grouped by tile plane I + J + K
  unsigned* tile_done;    // per tile: sweeps completed (only grows)
  unsigned long long* claim;   // work counter of the dataflow schedule (only grows)
  int ntx, nty, ntz, P;
  int maxit;
  int mode;               // HS_GS_FORWARD / BACKWARD / SYMMETRIC
  int check_every;
  double tol;
};


// Relative residual of x through the Jacobi form r_i = a_ii (x'_i - x_i),
// reduced over the grid.  Neighbours come straight from global memory (a
// residual is formed once per check_every sweeps, so no tile staging; this
// also frees the GS block from the tile engine's three-warp minimum).
template <typename T, int OPK, int NDIM>
__device__ bool gs_residual(const GsArgs<T>& a, T* /*sm*/, double* sh, double bb, double* rel) {
  const Geom& g = a.g;
  // blocks leave a batch at different times
  if (!grid_sync(a.cm.ctrl, a.cm.partials, sh)) return false;
  const T* bsrc = (OPK == OP_VARK) ? a.b : a.bD;
  const T* x = a.x;
  double acc[1] = {0.0};
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < g.N;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % g.nx);
    const int j = (int)((idx / g.nx) % g.ny);
    const int k = (int)(idx / g.plane);
    Nbr<T> nb;
    nb.c = __ldcg(x + idx);
    nb.w = i > 0 ? __ldcg(x + idx - 1) : T(0);
    nb.e = i + 1 < g.nx ? __ldcg(x + idx + 1) : T(0);
    nb.s = j > 0 ? __ldcg(x + idx - g.nx) : T(0);
    nb.n = j + 1 < g.ny ? __ldcg(x + idx + g.nx) : T(0);
    nb.b = (NDIM == 3 && k > 0) ? __ldcg(x + idx - g.plane) : T(0);
    nb.t = (NDIM == 3 && k + 1 < g.nz) ? __ldcg(x + idx + g.plane) : T(0);
    const OpRaw<T, OPK> o = op_fetch<T, OPK, NDIM>(a.cf, g, idx, i, j, k);
    T d = jacobi_apply<T, OPK, NDIM>(a.cf, o, nb, __ldcg(bsrc + idx)) - nb.c;
    if constexpr (OPK == OP_VARK) d = d / o.d;
    acc[0] += widen(d) * widen(d);
  }
  block_sum<1>(acc, sh);
  double rr[1];
  if (!grid_reduce<1>(a.cm.ctrl, a.cm.partials, acc, rr, sh)) return false;
  const double sc = (OPK == OP_VARK) ? 1.0 : a.dscale2;
  *rel = sqrt(rr[0] * sc / bb);
  return true;
}

// Jacobi-form update x_i = D_i (b_i + sum_j a_ij x_j) split in two: gs_old
// gathers the couplings to the neighbours not yet updated in this sweep (upper
// neighbours of a forward sweep, lower ones of a backward sweep) into the
// pre-scaled right-hand side, gs_new adds the already-updated neighbours (x
// one first: it is ready earliest) and applies D_i (variable coefficients;
// constant couplings come pre-divided by a_ii).
template <typename T, int OPK, int NDIM>
__device__ __forceinline__ T gs_old(const Coef<T>& cf, const OpRaw<T, OPK>& o, T bv, T vx, T vy, T vz, bool bw) {
  T cx, cy, cz;
  if constexpr (OPK == OP_VARK) {
    cx = bw ? o.xl : o.xu;
    cy = bw ? o.yl : o.yu;
    cz = bw ? o.zl : o.zu;
  } else {
    cx = bw ? cf.xl : cf.xu;
    cy = bw ? cf.yl : cf.yu;
    cz = bw ? cf.zl : cf.zu;
  }
  T y = fma(cx, vx, bv);
  y = fma(cy, vy, y);
  if (NDIM == 3) y = fma(cz, vz, y);
  return y;
}

template <typename T, int OPK, int NDIM>
__device__ __forceinline__ T gs_new(const Coef<T>& cf, const OpRaw<T, OPK>& o, T yold, T vx, T vy, T vz, bool bw) {
  T cx, cy, cz;
  if constexpr (OPK == OP_VARK) {
    cx = bw ? o.xu : o.xl;
    cy = bw ? o.yu : o.yl;
    cz = bw ? o.zu : o.zl;
  } else {
    cx = bw ? cf.xu : cf.xl;
    cy = bw ? cf.yu : cf.yl;
    cz = bw ? cf.zu : cf.zl;
  }
  T y = fma(cx, vx, yold);
  y = fma(cy, vy, y);
  if (NDIM == 3) y = fma(cz, vz, y);
  if constexpr (OPK == OP_VARK) y = y * o.d;
  return y;
}


// Warp 0 waits until every participating lane's sweep count *f has reached
// `target`, bounded by the solve's timeout (status DS_TIMEOUT); it ends early
// when another block has flagged an error.  All 32 lanes call it.
__device__ __forceinline__ bool gs_poll(bool mine, const unsigned* f, unsigned target, Ctrl* ctrl) {
  const int lane = threadIdx.x & 31;
  unsigned spins = 0;
  unsigned long long t0 = 0;
  while (true) {
    const bool sat = !mine || ld_acquire(f) >= target;
    if (__all_sync(0xffffffffu, sat)) return true;
    int stop = 0;
    if (lane == 0 && (++spins & 255) == 0) {
      if (t0 == 0) t0 = global_ns();
      if (ld_acquire_int(&ctrl->status) < 0) {
        stop = 1;
      } else if (global_ns() - t0 > ctrl->timeout_ns) {
        atomicCAS(&ctrl->status, 0, (int)DS_TIMEOUT);
        stop = 1;
      }
    }
    if (__shfl_sync(0xffffffffu, stop, 0)) return false;
  }
}


// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

// Constant couplings divided by the diagonal (the Jacobi form), 1 / a_ii and
// a_ii^2 (the residual's scale).
template <typename T>
static inline Coef<T> gs_jacobi_coef(const hs_op* A, T* invd, double* d2) {
  Coef<T> cf = {};
  ConstRow c = const_row(A);
  cf.xl = (T)(-c.xl / c.d);
  cf.xu = (T)(-c.xu / c.d);
  cf.yl = (T)(-c.yl / c.d);
  cf.yu = (T)(-c.yu / c.d);
  cf.zl = (T)(-c.zl / c.d);
  cf.zu = (T)(-c.zu / c.d);
  *invd = (T)(1.0 / c.d);
  *d2 = c.d * c.d;
  return cf;
}

// Initialises the control block and fills the fields of GsArgs that every
// schedule shares.  Variable coefficients: D = 1 / a_ii and the face
// couplings are formed into the arrays D, ax, ay, az carved by the caller.
template <typename T, int OPK>
static hs_status gs_setup(const SolveArgs& sa, const Common& cm, T* D, T* ax, T* ay, T* az, GsArgs<T>& a) {
  hs_status s = init_ctrl(cm, sa.o, sa.stream);
  if (s != HS_OK) return s;
  if constexpr (OPK == OP_VARK) {
    s = setup_vark(sa.A, sa.dtype, D, ax, ay, az, true, sa.stream);
    if (s != HS_OK) return s;
    a.cf.D = D;
    a.cf.ax = ax;
    a.cf.ay = ay;
    a.cf.az = az;
    a.dscale2 = 1.0;
  } else {
    a.cf = gs_jacobi_coef<T>(sa.A, &a.invd, &a.dscale2);
  }
  a.g = geom_of(sa.A);
  a.b = (const T*)sa.b;
  a.x = (T*)sa.x;
  a.cm = cm;
  a.maxit = sa.maxit;
  a.mode = sa.o.gs_mode;
  a.check_every = sa.o.check_every;
  a.tol = sa.tol;
  return HS_OK;
}

// After the launch: variable coefficients go back to the operator's own form
// for the true residual, the debug word of the calling translation unit is
// read, and the solve is finished (status, history, final residual).
template <typename T, int OPK>
static hs_status gs_finish(const SolveArgs& sa, const Common& cm, const GsArgs<T>& a, T* D, T* ax, T* ay, T* az,
                           hs_result* res, double* hist) {
  if (OPK == OP_VARK && sa.o.true_residual) {
    hs_status s = setup_vark(sa.A, sa.dtype, D, ax, ay, az, false, sa.stream);
    if (s != HS_OK) return s;
  }
  hs_status sd = hs_dbg_take(sa.stream);
  if (sd != HS_OK) return sd;
  return finish_solve_pub(sa, cm, D, ax, ay, az, a.bD, res, hist, sa.tol > 0.0);
}

// Tile count and tile planes of the larger tile table (hs_gs.cu); the other
// schedules keep the table's place in their workspace layout.
void gs_counts(const hs_op* A, int* ntiles, int* P);

// The pencil schedule (hs_gsp.cu).  gsp_applies: a 3-D Laplacian or upwind
// operator whose progress counts fit in 32 bits; gsp_fits: every pencil gets
// a resident warp of its own, with enough pencils to fill the GPU;
// gsp_progress_bytes: its workspace beyond b / a_ii.
bool gsp_applies(const SolveArgs& sa);
bool gsp_fits(const SolveArgs& sa);
size_t gsp_progress_bytes(const hs_op* A);
hs_status run_gs_pencils(const SolveArgs& sa, hs_result* res, double* hist);

// Small 1-/2-D grids on chip (hs_gs2d.cu): one block (gs2d) or one cluster
// of CTAs (gs2dc).
bool gs2d_applies(const SolveArgs& sa);
bool gs2dc_applies(const SolveArgs& sa);
hs_status run_gs2d(const SolveArgs& sa, hs_result* res, double* hist);
hs_status run_gs2dc(const SolveArgs& sa, hs_result* res, double* hist);

}  // namespace hs
