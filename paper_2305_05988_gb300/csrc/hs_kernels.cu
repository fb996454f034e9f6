// hs_kernels.cu -- stencil SpMV, residual, Jacobi, CG and BiCGStab kernels.
//
// The solver kernels are persistent cooperative kernels: one launch runs the
// whole iteration, with grid-wide reduce-barriers (hs_common.cuh) in place of
// the paper's MPI_Allreduce (section 3.3) and every vector update fused into
// the stencil pass that produces or consumes it.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <cmath>
#include <type_traits>

#include <vector>

#include "hs_internal.h"
#include "hs_krylov.cuh"

namespace hs {

// ===========================================================================
// SpMV and residual (one work item per block)
// ===========================================================================

template <typename T, int OPK, int NDIM>
__global__ void __launch_bounds__(512) k_spmv(Geom g, Tiling tl, Coef<T> cf, T sigma, const T* __restrict__ x,
                                              T* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  LoadSrc<T, false> src{x};
  SpmvSink<T, OPK, NDIM> sink{cf, g, sigma, y};
  for (int item = blockIdx.x; item < tl.items(); item += gridDim.x) zmarch_item<T, NDIM, cx_st<OPK>()>(g, tl, item, sm, src, sink);
}

template <typename T, int OPK, int NDIM>
__global__ void __launch_bounds__(512) k_residual(Geom g, Tiling tl, Coef<T> cf, T sigma, const T* __restrict__ b,
                                                  const T* __restrict__ x, T* __restrict__ r, double* partials) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double sh[32 * 2];
  T* sm = reinterpret_cast<T*>(smraw);
  LoadSrc<T, false> src{x};
  ResidualSink<T, OPK, NDIM> sink{cf, g, sigma, b, r, {0.0, 0.0}};
  for (int item = blockIdx.x; item < tl.items(); item += gridDim.x) zmarch_item<T, NDIM, cx_st<OPK>()>(g, tl, item, sm, src, sink);
  block_sum<2>(sink.acc, sh);
  if (partials && threadIdx.x == 0) {
    partials[2 * blockIdx.x] = sink.acc[0];
    partials[2 * blockIdx.x + 1] = sink.acc[1];
  }
}

// Sums nb x ns partials in block order (one block).
__global__ void k_finalize(const double* partials, int nb, int ns, double* out) {
  __shared__ double sh[32 * 2];
  double acc[2] = {0.0, 0.0};
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    acc[0] += partials[(size_t)b * ns];
    if (ns > 1) acc[1] += partials[(size_t)b * ns + 1];
  }
  block_sum<2>(acc, sh);
  if (threadIdx.x == 0) {
    out[0] = acc[0];
    if (ns > 1) out[1] = acc[1];
  }
}

// ===========================================================================
// Variable-coefficient setup: harmonic-mean face couplings from k.
// D = sum_f kappa_f / h_d^2 (or its inverse), a{x,y,z}_i = kappa of the lower
// face / h_d^2 (a boundary face uses kappa = k_i).
// ===========================================================================

__device__ __forceinline__ double harm(double a, double b) { return 2.0 * a * b / (a + b); }

template <typename T, typename K>
__global__ void k_vark_setup(Geom g, int ndim, const K* __restrict__ kk, double ihx, double ihy, double ihz,
                             T* D, T* ax, T* ay, T* az, int invert) {
  for (long long idx = gtid(); idx < g.N; idx += gstride()) {
    int i = (int)(idx % g.nx);
    int j = (int)((idx / g.nx) % g.ny);
    int k = (int)(idx / g.plane);
    double kc = (double)kk[idx];
    double d = 0.0;
    double lo, up;
    lo = (i > 0) ? harm(kc, (double)kk[idx - 1]) : kc;
    up = (i + 1 < g.nx) ? harm(kc, (double)kk[idx + 1]) : kc;
    d += lo * ihx;
    d += up * ihx;
    ax[idx] = (T)(lo * ihx);
    if (ndim >= 2) {
      lo = (j > 0) ? harm(kc, (double)kk[idx - g.nx]) : kc;
      up = (j + 1 < g.ny) ? harm(kc, (double)kk[idx + g.nx]) : kc;
      d += lo * ihy;
      d += up * ihy;
      ay[idx] = (T)(lo * ihy);
    } else {
      ay[idx] = T(0);
    }
    if (ndim >= 3) {
      lo = (k > 0) ? harm(kc, (double)kk[idx - g.plane]) : kc;
      up = (k + 1 < g.nz) ? harm(kc, (double)kk[idx + g.plane]) : kc;
      d += lo * ihz;
      d += up * ihz;
      az[idx] = (T)(lo * ihz);
    } else if (az) {
      az[idx] = T(0);
    }
    D[idx] = invert ? (T)(1.0 / d) : (T)d;
  }
}

// ===========================================================================
// Jacobi (section 3.1), out of place, persistent.
// ===========================================================================

template <typename T>
struct JacArgs {
  Geom g;
  Tiling tl;
  Coef<T> cf;      // constant: g = -a/a_ii couplings; variable: D = 1/a_ii
  T invd;          // constant: 1/a_ii
  double dscale2;  // constant: a_ii^2 (residual = a_ii (x' - x))
  const T* b;
  T* bD;           // workspace b/a_ii (constant coefficients)
  T* x0;           // caller's x
  T* x1;           // workspace ping-pong buffer
  Common cm;
  int maxit;
  double tol;
  int fuse;        // 1: fuse the residual of each iterate into the next sweep
};

// x' = Jacobi update of x; with FUSE also accumulates the residual of x,
// r = a_ii (x' - x).  FUSE is a template parameter: a run-time flag lets the
// compiler predicate the residual arithmetic, which then still issues on the
// FP64 pipe for every node.
template <typename T, int OPK, int NDIM, bool FUSE>
struct JacobiSink {
  static constexpr bool kBox = OPK == OP_BOX27;
  Coef<T> cf;
  Geom g;
  const T* bsrc;   // b/a_ii (constant) or b (variable)
  T* xd;
  double acc[1];
  struct Raw {
    OpRaw<T, OPK> o;
    T b;
  };
  __device__ __forceinline__ Raw fetch(long long idx, int i, int j, int k) const {
    return Raw{op_fetch<T, OPK, NDIM>(cf, g, idx, i, j, k), __ldcg(bsrc + idx)};
  }
  __device__ __forceinline__ void operator()(long long idx, const Nbr<T>& nb, const Raw& q, int, int, int) {
    T xn = jacobi_apply<T, OPK, NDIM>(cf, q.o, nb, q.b);
    xd[idx] = xn;
    if constexpr (FUSE) {
      T d = xn - nb.c;
      if constexpr (OPK == OP_VARK) d = d / q.o.d;
      acc[0] += widen(d) * widen(d);
    }
  }
};

template <typename T, int OPK, int NDIM, bool FUSE>
__global__ void __launch_bounds__(512) k_jacobi(JacArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double sh[32 * MAX_SCAL];
  T* sm = reinterpret_cast<T*>(smraw);
  const long long N = a.g.N;

  double acc[1] = {0.0};
  for (long long i = gtid(); i < N; i += gstride()) {
    T bv = a.b[i];
    if (OPK != OP_VARK) a.bD[i] = bv * a.invd;
    acc[0] += widen(bv) * widen(bv);
  }
  block_sum<1>(acc, sh);
  double bb[1];
  if (!grid_reduce<1>(a.cm.ctrl, a.cm.partials, acc, bb, sh)) return;
  if (bb[0] == 0.0) {
    for (long long i = gtid(); i < N; i += gstride()) a.x0[i] = T(0);
    finish(a.cm.ctrl, DS_CONVERGED, 0, 0.0);
    return;
  }
  const T* bsrc = (OPK == OP_VARK) ? a.b : a.bD;
  T* xs = a.x0;
  T* xd = a.x1;
  int iters = 0, status = DS_CONVERGED;
  double rel = -1.0;
  for (int k = 0;; k++) {
    if (!FUSE && k == a.maxit) {
      iters = k;
      break;
    }
    LoadSrc<T, true> src{xs};
    JacobiSink<T, OPK, NDIM, FUSE> sink{a.cf, a.g, bsrc, xd, {0.0}};
    for (int pos = blockIdx.x; pos < a.tl.items(); pos += gridDim.x)
      zmarch_item<T, NDIM, (cx_jac<T, OPK>())>(a.g, a.tl, pos, sm, src, sink);
    if constexpr (FUSE) {
      block_sum<1>(sink.acc, sh);
      double rr[1];
      if (!grid_reduce<1>(a.cm.ctrl, a.cm.partials, sink.acc, rr, sh)) return;
      double sc = (OPK == OP_VARK) ? 1.0 : a.dscale2;
      rel = sqrt(rr[0] * sc / bb[0]);
      if (blockIdx.x == 0 && threadIdx.x == 0) a.cm.hist[k] = rel;
      if (!finite_d(rel)) {
        iters = k;
        status = DS_NONFINITE;
        break;
      }
      if (rel <= a.tol || k == a.maxit) {
        iters = k;
        status = (rel <= a.tol) ? DS_CONVERGED : DS_MAXIT;
        break;
      }
    } else {
      if (!grid_sync(a.cm.ctrl, a.cm.partials, sh)) return;
    }
    T* t = xs;
    xs = xd;
    xd = t;
  }
  if (xs != a.x0) {
    for (long long i = gtid(); i < N; i += gstride()) a.x0[i] = ldcg(xs + i);
  }
  finish(a.cm.ctrl, status, iters, rel);
}

// Register caps of the persistent solver kernels (0: compiler's choice) and
// the CG x-deferral.  Defaults from A/B runs on GB300 at 256^3: FP64 CG on a
// constant-coefficient operator 421 -> 410 us/iteration with the x update
// deferred and 64 registers (either alone is slower: 441 / 433); FP64
// BiCGStab 890 -> 859 us/iteration at 80 registers (3 blocks of 256 threads
// per SM); the deferral slows FP64 variable-coefficient CG (1.43 -> 1.50 s),
// which keeps the classical pass 2.  Override with -DHS_CG_MAXNREG=... etc.
#ifndef HS_CG_MAXNREG
#define HS_CG_MAXNREG 64
#endif
#ifndef HS_CG_XDEFER
#define HS_CG_XDEFER 1
#endif
#ifndef HS_BI_MAXNREG
#define HS_BI_MAXNREG 80
#endif
// FP32 CG on the variable-coefficient operator (the inner solve of mixed
// refinement): 64 registers, four blocks per SM instead of three (512^3:
// 1.74 -> 1.63 ms/iteration; 48 or 40 spill and run at 2.1-2.2 ms; the
// FP32 Laplacian is slower under the cap, 1.29 -> 1.59, and keeps none).
#ifndef HS_CG32_MAXNREG
#define HS_CG32_MAXNREG 64
#endif
// FP64 CG on the variable-coefficient operator: 80 registers (512^3: 3.73 ->
// 3.49 ms/iteration; 64 spills, 4.37).  FP32 BiCGStab: 64 registers, four
// blocks per SM instead of two (512^3 upwind 3.63 -> 2.44, diffusion 4.24 ->
// 3.23 ms/iteration; 80: 2.64 / 3.39).
#ifndef HS_CGV64_MAXNREG
#define HS_CGV64_MAXNREG 80
#endif
#ifndef HS_BI32_MAXNREG
#define HS_BI32_MAXNREG 64
#endif
template <typename T, int OPK>
constexpr int cg_maxnreg() {
  if (sizeof(T) == 4) return (HS_CG32_MAXNREG > 0 && OPK == OP_VARK) ? HS_CG32_MAXNREG : 255;
  if (OPK == OP_VARK) return HS_CGV64_MAXNREG > 0 ? HS_CGV64_MAXNREG : 255;
  return HS_CG_MAXNREG > 0 ? HS_CG_MAXNREG : 255;
}
template <typename T, int OPK>
constexpr int bi_maxnreg() {
  if (sizeof(T) == 4) return HS_BI32_MAXNREG > 0 ? HS_BI32_MAXNREG : 255;
  return HS_BI_MAXNREG > 0 ? HS_BI_MAXNREG : 255;
}

template <typename T, int OPK, int NDIM>
__global__ void __launch_bounds__(512) __maxnreg__((cg_maxnreg<T, OPK>())) k_cg(CgArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double sh[32 * MAX_SCAL];
  const Team tm = grid_team(a.cm.ctrl, a.cm.partials);
  constexpr bool xdefer = HS_CG_XDEFER && sizeof(T) == 8 && OPK != OP_VARK;
  team_finish(tm, cg_body<T, OPK, NDIM, cx_cg<T, OPK>(), xdefer>(a, tm, reinterpret_cast<T*>(smraw), sh));
}

template <typename T, int OPK, int NDIM>
__global__ void __launch_bounds__(512) __maxnreg__((bi_maxnreg<T, OPK>())) k_bicgstab(BiArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double sh[32 * MAX_SCAL];
  const Team tm = grid_team(a.cm.ctrl, a.cm.partials);
  team_finish(tm, bicgstab_body<T, OPK, NDIM>(a, tm, reinterpret_cast<T*>(smraw), sh));
}

// ===========================================================================
// Host side: coefficients, launch shapes, dispatch.
// ===========================================================================

__global__ void k_init_ctrl(Ctrl* c, unsigned long long timeout_ns) {
  if (threadIdx.x == 0) {
    c->count = 0;
    c->gen = 0;
    c->status = 0;
    c->iters = 0;
    c->restarts = 0;
    c->timeout_ns = timeout_ns;
    c->rel_res = -1.0;
  }
}

static int g_sm_count = -1;
int sm_count() {
  if (g_sm_count < 0) {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    g_sm_count = n > 0 ? n : 1;
  }
  return g_sm_count;
}

Tiling choose_tiling(const Geom& g, int by, int grid, bool src_expensive, int planes, int cx) {
  Tiling t;
  t.by = by;
  t.cx = cx;
  t.tiles_x = (g.nx + BX * cx - 1) / (BX * cx);
  t.tiles_y = (g.ny + by - 1) / by;
  const int txy = t.tiles_x * t.tiles_y;
  if (g.nz == 1) {
    t.chunks = 1;
    t.lz = 1;
    return t;
  }
  if (planes > 0) {
    t.lz = std::min(g.nz, planes);
    t.chunks = (g.nz + t.lz - 1) / t.lz;
    return t;
  }
  if (grid <= 0) {
    t.lz = std::min(g.nz, 32);
    t.chunks = (g.nz + t.lz - 1) / t.lz;
    return t;
  }
  const double over = src_expensive ? 2.0 : 1.0;
  double best = 1e300;
  int best_lz = g.nz;
  for (int lz = 4; lz <= g.nz; lz++) {
    int chunks = (g.nz + lz - 1) / lz;
    if (lz > 4 && (g.nz + lz - 2) / (lz - 1) == chunks) continue;  // same chunk count, smaller lz better
    long long items = (long long)txy * chunks;
    long long waves = (items + grid - 1) / grid;
    double cost = (double)waves * (lz + over);
    if (cost < best - 1e-9) {
      best = cost;
      best_lz = lz;
    }
  }
  if (g.nz < 4) best_lz = g.nz;
  t.lz = best_lz;
  t.chunks = (g.nz + t.lz - 1) / t.lz;
  return t;
}

ConstRow const_row(const hs_op* A) {
  ConstRow c = {0, 0, 0, 0, 0, 0, 0};
  if (A->kind == KIND_HPCG7 || A->kind == KIND_HPCG27) {
    // every coupling -1, diagonal 27 (the 27-point kernels read only d and
    // the x coupling, see scaled_coef and jacobi_coef)
    c.d = 27.0;
    double* cs[6] = {&c.xl, &c.xu, &c.yl, &c.yu, &c.zl, &c.zu};
    for (int q = 0; q < 2 * A->ndim; q++) *cs[q] = -1.0;
    return c;
  }
  double* lo[3] = {&c.xl, &c.yl, &c.zl};
  double* up[3] = {&c.xu, &c.yu, &c.zu};
  for (int d = 0; d < A->ndim; d++) {
    double ih2 = 1.0 / (A->h[d] * A->h[d]);
    double bh = (A->kind == KIND_UPWIND) ? A->beta[d] / A->h[d] : 0.0;
    *lo[d] = -ih2 - bh;
    *up[d] = -ih2;
    c.d += 2.0 * ih2 + bh;
  }
  return c;
}

// Jacobi coefficients g = -a/a_ii.
template <typename T>
static Coef<T> jacobi_coef(const hs_op* A, T* invd, double* d2) {
  Coef<T> cf = {};
  ConstRow c = const_row(A);
  cf.d = (T)0;
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

size_t vark_coef_bytes(const hs_op* A, hs_dtype dt) {
  if (A->kind != KIND_DIFFUSION) return 0;
  size_t N = (size_t)(A->n[0] * A->n[1] * A->n[2]);
  size_t es = dt == HS_F64 ? 8 : 4;
  return 4 * ((N * es + 255) & ~(size_t)255);
}

hs_status setup_vark(const hs_op* A, hs_dtype dt, void* D, void* ax, void* ay, void* az, bool invert_diag,
                     cudaStream_t st) {
  Geom g = geom_of(A);
  double ih[3];
  for (int d = 0; d < 3; d++) ih[d] = d < A->ndim ? 1.0 / (A->h[d] * A->h[d]) : 0.0;
  int blocks = (int)std::min<long long>((g.N + 255) / 256, (long long)sm_count() * 16);
  if (blocks < 1) blocks = 1;
  if (dt == HS_F64) {
    if (A->kdt == HS_F64)
      k_vark_setup<double, double><<<blocks, 256, 0, st>>>(g, A->ndim, (const double*)A->k, ih[0], ih[1], ih[2],
                                                           (double*)D, (double*)ax, (double*)ay, (double*)az,
                                                           invert_diag);
    else
      k_vark_setup<double, float><<<blocks, 256, 0, st>>>(g, A->ndim, (const float*)A->k, ih[0], ih[1], ih[2],
                                                          (double*)D, (double*)ax, (double*)ay, (double*)az,
                                                          invert_diag);
  } else {
    if (A->kdt == HS_F64)
      k_vark_setup<float, double><<<blocks, 256, 0, st>>>(g, A->ndim, (const double*)A->k, ih[0], ih[1], ih[2],
                                                          (float*)D, (float*)ax, (float*)ay, (float*)az,
                                                          invert_diag);
    else
      k_vark_setup<float, float><<<blocks, 256, 0, st>>>(g, A->ndim, (const float*)A->k, ih[0], ih[1], ih[2],
                                                         (float*)D, (float*)ax, (float*)ay, (float*)az,
                                                         invert_diag);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HS_OK : cuda_fail(e, "variable-coefficient setup launch");
}

// ---- dispatch over (element type, operator kind, dimensionality) ---------
template <typename T_, int OPK_, int NDIM_>
struct Tag {
  using T = T_;
  static constexpr int OPK = OPK_;
  static constexpr int NDIM = NDIM_;
};

template <class F>
static hs_status dispatch(hs_dtype dt, int opk, int ndim, F&& f) {
  const int nd = ndim >= 3 ? 3 : 2;
#define HS_CASE(TT, OK, ND) \
  if (opk == OK && nd == ND) return f(Tag<TT, OK, ND>{});
  if (dt == HS_F64) {
    HS_CASE(double, OP_SYM, 2)
    HS_CASE(double, OP_SYM, 3)
    HS_CASE(double, OP_NONSYM, 2)
    HS_CASE(double, OP_NONSYM, 3)
    HS_CASE(double, OP_VARK, 2)
    HS_CASE(double, OP_VARK, 3)
    HS_CASE(double, OP_BOX27, 3)
  } else {
    HS_CASE(float, OP_SYM, 2)
    HS_CASE(float, OP_SYM, 3)
    HS_CASE(float, OP_NONSYM, 2)
    HS_CASE(float, OP_NONSYM, 3)
    HS_CASE(float, OP_VARK, 2)
    HS_CASE(float, OP_VARK, 3)
    HS_CASE(float, OP_BOX27, 3)
  }
#undef HS_CASE
  set_error("unsupported operator / dtype combination");
  return HS_ERR_INVALID;
}

// Variable-coefficient SpMV without a workspace: face couplings are formed
// on the fly from k (harmonic means), y_i = sum_f kappa_f (x_i - x_j) / h^2.
template <typename T, typename K, int NDIM>
struct VarkDirectSink {
  Geom g;
  const K* kk;
  double ihx, ihy, ihz;
  T* y;
  struct Raw {};
  __device__ __forceinline__ Raw fetch(long long, int, int, int) const { return Raw{}; }
  __device__ __forceinline__ void operator()(long long idx, const Nbr<T>& nb, const Raw&, int i, int j, int k) {
    const double kc = (double)__ldg(kk + idx), xc = (double)nb.c;
    double acc = 0.0;
    double kap;
    kap = (i > 0) ? harm(kc, (double)__ldg(kk + idx - 1)) : kc;
    acc += kap * ihx * (xc - (double)nb.w);
    kap = (i + 1 < g.nx) ? harm(kc, (double)__ldg(kk + idx + 1)) : kc;
    acc += kap * ihx * (xc - (double)nb.e);
    if (ihy != 0.0) {
      kap = (j > 0) ? harm(kc, (double)__ldg(kk + idx - g.nx)) : kc;
      acc += kap * ihy * (xc - (double)nb.s);
      kap = (j + 1 < g.ny) ? harm(kc, (double)__ldg(kk + idx + g.nx)) : kc;
      acc += kap * ihy * (xc - (double)nb.n);
    }
    if (NDIM == 3) {
      kap = (k > 0) ? harm(kc, (double)__ldg(kk + idx - g.plane)) : kc;
      acc += kap * ihz * (xc - (double)nb.b);
      kap = (k + 1 < g.nz) ? harm(kc, (double)__ldg(kk + idx + g.plane)) : kc;
      acc += kap * ihz * (xc - (double)nb.t);
    }
    y[idx] = (T)acc;
  }
};

template <typename T, typename K, int NDIM>
__global__ void __launch_bounds__(512) k_spmv_vark_direct(Geom g, Tiling tl, const K* __restrict__ kk, double ihx,
                                                          double ihy, double ihz, const T* __restrict__ x,
                                                          T* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  LoadSrc<T, false> src{x};
  VarkDirectSink<T, K, NDIM> sink{g, kk, ihx, ihy, ihz, y};
  for (int item = blockIdx.x; item < tl.items(); item += gridDim.x) zmarch_item<T, NDIM, CX_ST>(g, tl, item, sm, src, sink);
}

// r = b - y (elementwise), used by the residual of diffusion operators.
template <typename T>
__global__ void k_sub_from(const T* __restrict__ b, T* __restrict__ r, long long N) {
  for (long long i = gtid(); i < N; i += gstride()) r[i] = b[i] - r[i];
}

template <typename T, int NDIM>
static hs_status spmv_vark_direct(const hs_op* A, const void* x, void* y, cudaStream_t st) {
  Geom g = geom_of(A);
  int by = rows_per_tile(g);
  Tiling tl = choose_tiling(g, by, 0, false, 0, CX_ST);
  double ih[3];
  for (int d = 0; d < 3; d++) ih[d] = d < A->ndim ? 1.0 / (A->h[d] * A->h[d]) : 0.0;
  if (A->kdt == HS_F64)
    k_spmv_vark_direct<T, double, NDIM><<<tl.items(), 32 * by, slab_bytes<T>(by, CX_ST), st>>>(
        g, tl, (const double*)A->k, ih[0], ih[1], ih[2], (const T*)x, (T*)y);
  else
    k_spmv_vark_direct<T, float, NDIM><<<tl.items(), 32 * by, slab_bytes<T>(by, CX_ST), st>>>(
        g, tl, (const float*)A->k, ih[0], ih[1], ih[2], (const T*)x, (T*)y);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HS_OK : cuda_fail(e, "spmv launch");
}

hs_status run_spmv(const hs_op* A, hs_dtype dt, const void* x, void* y, cudaStream_t st) {
  Geom g = geom_of(A);
  return dispatch(dt, opkind_of(A), A->ndim, [&](auto tag) -> hs_status {
    using Tg = decltype(tag);
    using T = typename Tg::T;
    constexpr int OPK = Tg::OPK, NDIM = Tg::NDIM;
    if (OPK == OP_VARK) return spmv_vark_direct<T, NDIM>(A, x, y, st);
    double sigma;
    Coef<T> cf = op_coef<T>(A, nullptr, nullptr, nullptr, nullptr, &sigma);
    int by = rows_per_tile(g);
    Tiling tl = choose_tiling(g, by, 0, false, 0, cx_st<OPK>());
    k_spmv<T, OPK, NDIM><<<tl.items(), 32 * by, slab_bytes<T>(by, cx_st<OPK>()), st>>>(g, tl, cf, (T)sigma, (const T*)x, (T*)y);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? hs_dbg_take(st) : cuda_fail(e, "spmv launch");
  });
}

hs_status run_residual_plain(const hs_op* A, hs_dtype dt, const void* b, const void* x, void* r, cudaStream_t st) {
  Geom g = geom_of(A);
  if (A->kind == KIND_DIFFUSION) {
    hs_status s = run_spmv(A, dt, x, r, st);
    if (s != HS_OK) return s;
    int blocks = (int)std::min<long long>((g.N + 255) / 256, (long long)sm_count() * 16);
    if (blocks < 1) blocks = 1;
    if (dt == HS_F64)
      k_sub_from<double><<<blocks, 256, 0, st>>>((const double*)b, (double*)r, g.N);
    else
      k_sub_from<float><<<blocks, 256, 0, st>>>((const float*)b, (float*)r, g.N);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? hs_dbg_take(st) : cuda_fail(e, "residual launch");
  }
  return dispatch(dt, opkind_of(A), A->ndim, [&](auto tag) -> hs_status {
    using Tg = decltype(tag);
    using T = typename Tg::T;
    constexpr int OPK = Tg::OPK, NDIM = Tg::NDIM;
    if (OPK == OP_VARK) return HS_ERR_INVALID;
    double sigma;
    Coef<T> cf = op_coef<T>(A, nullptr, nullptr, nullptr, nullptr, &sigma);
    int by = rows_per_tile(g);
    Tiling tl = choose_tiling(g, by, 0, false, 0, cx_st<OPK>());
    k_residual<T, OPK, NDIM><<<tl.items(), 32 * by, slab_bytes<T>(by, cx_st<OPK>()), st>>>(g, tl, cf, (T)sigma, (const T*)b,
                                                                               (const T*)x, (T*)r, nullptr);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? hs_dbg_take(st) : cuda_fail(e, "residual launch");
  });
}

// r = b - A x with the solver's coefficient arrays, plus ||r||^2, ||b||^2
// reduced deterministically into norms_dev[0..1] (partials: >= grid*2 doubles).
static hs_status residual_norms(const hs_op* A, hs_dtype dt, const void* D, const void* ax, const void* ay,
                                const void* az, const void* b, const void* x, void* r, double* norms_dev,
                                double* partials_dev, cudaStream_t st) {
  Geom g = geom_of(A);
  return dispatch(dt, opkind_of(A), A->ndim, [&](auto tag) -> hs_status {
    using Tg = decltype(tag);
    using T = typename Tg::T;
    constexpr int OPK = Tg::OPK, NDIM = Tg::NDIM;
    double sigma;
    Coef<T> cf = op_coef<T>(A, D, ax, ay, az, &sigma);
    int by = rows_per_tile(g);
    constexpr int cx = cx_st<OPK>();   // must match the kernel's columns per lane
    Tiling tl = choose_tiling(g, by, 0, false, 0, cx);
    int grid = std::min(tl.items(), MAX_BLOCKS * MAX_SCAL / 2);
    k_residual<T, OPK, NDIM><<<grid, 32 * by, slab_bytes<T>(by, cx), st>>>(g, tl, cf, (T)sigma, (const T*)b,
                                                                        (const T*)x, (T*)r, partials_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "residual launch");
    k_finalize<<<1, 256, 0, st>>>(partials_dev, grid, 2, norms_dev);
    e = cudaGetLastError();
    return e == cudaSuccess ? HS_OK : cuda_fail(e, "finalize launch");
  });
}

hs_status launch_coop(const void* fn, int grid, int block, void** args, size_t smem, cudaStream_t st) {
  cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, smem, st);
  if (e != cudaSuccess) return cuda_fail(e, "cooperative launch");
  return HS_OK;
}

// One block of a team of two: the reduce-barrier waits for a block that is
// never launched and must give up with DS_TIMEOUT.
__global__ void k_diag_team(Ctrl* ctrl, double* partials) {
  __shared__ double sh[32 * MAX_SCAL];
  Team tm;
  tm.rank = 0;
  tm.size = 2;
  tm.ctrl = ctrl;
  tm.partials = partials;
  double z[1] = {0.0}, o[1];
  team_reduce<1>(tm, z, o, sh);
}

hs_status diag_team_wait(Ctrl* ctrl, double* partials, cudaStream_t st) {
  k_diag_team<<<1, 128, 0, st>>>(ctrl, partials);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HS_OK : cuda_fail(e, "diagnostic launch");
}

hs_status init_ctrl(const Common& cm, const hs_opts& o, cudaStream_t st) {
  double t = o.timeout_s > 0 ? o.timeout_s : 2.0;
  k_init_ctrl<<<1, 32, 0, st>>>(cm.ctrl, (unsigned long long)(t * 1e9));
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HS_OK : cuda_fail(e, "control init");
}

// Common solver tail: optional true residual of the returned x into
// ctrl->aux[0..1], then read back the control block and history.
struct Tail {
  const hs_op* A;
  hs_dtype dt;
  const void *D, *ax, *ay, *az;   // coefficient arrays (diffusion) or null
  const void* b;
  const void* x;
  void* rbuf;                     // scratch vector of N elements
};

// The asynchronous tail: the control block becomes an hs_result in device
// memory and the history is copied device to device, all on the stream.
__global__ void k_finalize_dev(const Ctrl* c, int maxit, int true_res, int want_hist, const double* hsrc,
                               double* hdst, hs_result* out) {
  const int iters = c->iters;
  if (threadIdx.x == 0 && out) {
    hs_result r;
    r.iters = iters;
    r.rel_res = c->rel_res;
    r.restarts = c->restarts;
    r.outer = 0;
    r.inner_iters = 0;
    r.true_rel_res = -1.0;
    if (true_res) {
      const double rr = c->aux[0], bb = c->aux[1];
      r.true_rel_res = bb > 0.0 ? sqrt(rr / bb) : 0.0;
      if (r.rel_res < 0.0) r.rel_res = r.true_rel_res;
    }
    switch (c->status) {
      case DS_CONVERGED: r.status = HS_OK; break;
      case DS_MAXIT: r.status = HS_NOT_CONVERGED; break;
      case DS_BREAKDOWN: r.status = HS_ERR_BREAKDOWN; break;
      case DS_NONFINITE: r.status = HS_ERR_NONFINITE; break;
      case DS_TIMEOUT: r.status = HS_ERR_TIMEOUT; break;
      default: r.status = HS_ERR_CUDA; break;
    }
    *out = r;
  }
  if (hdst && want_hist) {
    const int n = (iters < maxit ? iters : maxit) + 1;
    for (int q = threadIdx.x; q < n; q += blockDim.x) hdst[q] = hsrc[q];
  }
}

static hs_status finish_solve(const SolveArgs& sa, const Common& cm, const Tail& t, hs_result* res, double* hist,
                              bool want_hist) {
  {
    hs_status sd = hs_dbg_take(sa.stream);
    if (sd != HS_OK) return sd;
  }
  if (sa.async_dev) {
    if (sa.o.true_residual) {
      hs_status s = residual_norms(t.A, t.dt, t.D, t.ax, t.ay, t.az, t.b, t.x, t.rbuf, &cm.ctrl->aux[0], cm.partials,
                                   sa.stream);
      if (s != HS_OK) return s;
    }
    k_finalize_dev<<<1, 256, 0, sa.stream>>>(cm.ctrl, sa.maxit, sa.o.true_residual ? 1 : 0, want_hist ? 1 : 0, cm.hist,
                                             sa.hist_dev, sa.res_dev);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HS_OK : cuda_fail(e, "result kernel");
  }
  if (sa.o.true_residual) {
    hs_status s = residual_norms(t.A, t.dt, t.D, t.ax, t.ay, t.az, t.b, t.x, t.rbuf, &cm.ctrl->aux[0], cm.partials,
                                 sa.stream);
    if (s != HS_OK) return s;
  }
  Ctrl h;
  cudaError_t e = cudaMemcpyAsync(&h, cm.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, sa.stream);
  if (e != cudaSuccess) return cuda_fail(e, "control read-back");
  e = cudaStreamSynchronize(sa.stream);
  if (e != cudaSuccess) return cuda_fail(e, "solver kernel");
  if (hist && want_hist) {
    int n = std::min(h.iters, sa.maxit) + 1;
    if (n > 0) {
      e = cudaMemcpy(hist, cm.hist, sizeof(double) * n, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(e, "history read-back");
    }
  }
  res->iters = h.iters;
  res->rel_res = h.rel_res;
  res->restarts = h.restarts;
  res->true_rel_res = -1.0;
  if (sa.o.true_residual) {
    double rr = h.aux[0], bb = h.aux[1];
    res->true_rel_res = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    if (res->rel_res < 0.0) res->rel_res = res->true_rel_res;
  }
  switch (h.status) {
    case DS_CONVERGED: res->status = HS_OK; break;
    case DS_MAXIT: res->status = HS_NOT_CONVERGED; break;
    case DS_BREAKDOWN: res->status = HS_ERR_BREAKDOWN; break;
    case DS_NONFINITE: res->status = HS_ERR_NONFINITE; break;
    case DS_TIMEOUT: res->status = HS_ERR_TIMEOUT; break;
    default:
      res->status = HS_ERR_CUDA;
      set_error("solver ended without a status (%d)", h.status);
      return HS_ERR_CUDA;
  }
  if (res->status == HS_ERR_TIMEOUT) set_error("a device-side wait ran out (timeout)");
  if (res->status == HS_ERR_BREAKDOWN) set_error("Krylov breakdown (vanishing denominator)");
  if (res->status == HS_ERR_NONFINITE) set_error("non-finite value in a reduction");
  return (hs_status)res->status;
}

hs_status finish_solve_pub(const SolveArgs& sa, const Common& cm, const void* D, const void* ax, const void* ay,
                           const void* az, void* rbuf, hs_result* res, double* hist, bool want_hist) {
  Tail t{sa.A, sa.dtype, D, ax, ay, az, sa.b, sa.x, rbuf};
  return finish_solve(sa, cm, t, res, hist, want_hist);
}

// ---- Jacobi -----------------------------------------------------------------
hs_status run_jacobi(const SolveArgs& sa, hs_result* res, double* hist) {
  if (jacobi_tb_applies(sa)) return run_jacobi_tb(sa, res, hist);
  return dispatch(sa.dtype, opkind_of(sa.A), sa.A->ndim, [&](auto tag) -> hs_status {
    using Tg = decltype(tag);
    using T = typename Tg::T;
    constexpr int OPK = Tg::OPK, NDIM = Tg::NDIM;
    const hs_op* A = sa.A;
    Geom g = geom_of(A);
    Carve c{sa.ws, 0, sa.ws_bytes, true};
    Common cm = carve_common(c, sa.maxit);
    JacArgs<T> a = {};
    a.x1 = c.take<T>(g.N);
    a.bD = c.take<T>(g.N);
    T *D = nullptr, *ax = nullptr, *ay = nullptr, *az = nullptr;
    if (OPK == OP_VARK) {
      D = c.take<T>(g.N);
      ax = c.take<T>(g.N);
      ay = c.take<T>(g.N);
      az = c.take<T>(g.N);
    }
    if (!c.ok) {
      set_error("workspace too small for Jacobi");
      return HS_ERR_WORKSPACE;
    }
    hs_status s = init_ctrl(cm, sa.o, sa.stream);
    if (s != HS_OK) return s;
    if (OPK == OP_VARK) {
      s = setup_vark(A, sa.dtype, D, ax, ay, az, true, sa.stream);
      if (s != HS_OK) return s;
      a.cf.D = D;
      a.cf.ax = ax;
      a.cf.ay = ay;
      a.cf.az = az;
      a.dscale2 = 1.0;
    } else {
      a.cf = jacobi_coef<T>(A, &a.invd, &a.dscale2);
    }
    a.g = g;
    a.b = (const T*)sa.b;
    a.x0 = (T*)sa.x;
    a.cm = cm;
    a.maxit = sa.maxit;
    a.tol = sa.tol;
    a.fuse = sa.tol > 0.0 ? 1 : 0;
    int by = rows_for(g, sa.o);
    constexpr int cx = cx_jac<T, OPK>();
    size_t smem = slab_bytes<T>(by, cx);
    int grid = 0;
    const void* kern = a.fuse ? (const void*)k_jacobi<T, OPK, NDIM, true> : (const void*)k_jacobi<T, OPK, NDIM, false>;
    s = a.fuse ? plan_persistent(k_jacobi<T, OPK, NDIM, true>, 32 * by, smem, g, by, false, &grid, &a.tl, sa.o, cx)
               : plan_persistent(k_jacobi<T, OPK, NDIM, false>, 32 * by, smem, g, by, false, &grid, &a.tl, sa.o, cx);
    if (s != HS_OK) return s;
    void* args[] = {&a};
    s = launch_coop(kern, grid, 32 * by, args, smem, sa.stream);
    if (s != HS_OK) return s;
    if (OPK == OP_VARK && sa.o.true_residual) {
      s = setup_vark(A, sa.dtype, D, ax, ay, az, false, sa.stream);  // un-inverted diagonal
      if (s != HS_OK) return s;
    }
    Tail t{A, sa.dtype, D, ax, ay, az, sa.b, sa.x, a.x1};
    return finish_solve(sa, cm, t, res, hist, sa.tol > 0.0);
  });
}

// ---- Krylov cores: launch one persistent solve on given coefficients --------
template <typename T, int OPK, int NDIM>
static hs_status cg_core(const hs_op* A, const Coef<T>& cf, double sigma, const T* b, T* x, double tol, int maxit,
                         const Common& cm, T* r, T* p0, T* p1, T* w, const hs_opts& o, cudaStream_t st) {
  CgArgs<T> a = {};
  a.g = geom_of(A);
  a.cf = cf;
  a.sigma = sigma;
  a.b = b;
  a.x = x;
  a.r = r;
  a.p0 = p0;
  a.p1 = p1;
  a.w = w;
  a.cm = cm;
  a.maxit = maxit;
  a.tol = tol;
  hs_status s = init_ctrl(cm, o, st);
  if (s != HS_OK) return s;
  int by = rows_for(a.g, o);
  constexpr int cx = cx_cg<T, OPK>();
  size_t smem = slab_bytes<T>(by, cx);
  int grid = 0;
  s = plan_persistent(k_cg<T, OPK, NDIM>, 32 * by, smem, a.g, by, true, &grid, &a.tl, o, cx);
  if (s != HS_OK) return s;
  void* args[] = {&a};
  return launch_coop((const void*)k_cg<T, OPK, NDIM>, grid, 32 * by, args, smem, st);
}

template <typename T, int OPK, int NDIM>
static hs_status bicgstab_core(const hs_op* A, const Coef<T>& cf, double sigma, const T* b, T* x, double tol,
                               int maxit, const Common& cm, T* const v[8], const hs_opts& o, cudaStream_t st,
                               double* trace = nullptr) {
  BiArgs<T> a = {};
  a.trace = trace;
  a.g = geom_of(A);
  a.cf = cf;
  a.sigma = sigma;
  a.b = b;
  a.x = x;
  a.r = v[0];
  a.rs = v[1];
  a.p0 = v[2];
  a.p1 = v[3];
  a.v0 = v[4];
  a.v1 = v[5];
  a.s = v[6];
  a.t = v[7];
  a.cm = cm;
  a.paper_order = o.paper_order;
  a.maxit = maxit;
  a.tol = tol;
  a.reps = o.restart_eps;
  hs_status s = init_ctrl(cm, o, st);
  if (s != HS_OK) return s;
  int by = rows_for(a.g, o);
  size_t smem = slab_bytes<T>(by, CX_BI);
  int grid = 0;
  s = plan_persistent(k_bicgstab<T, OPK, NDIM>, 32 * by, smem, a.g, by, true, &grid, &a.tl, o, CX_BI);
  if (s != HS_OK) return s;
  void* args[] = {&a};
  return launch_coop((const void*)k_bicgstab<T, OPK, NDIM>, grid, 32 * by, args, smem, st);
}

// ---- CG -----------------------------------------------------------------------
hs_status run_cg(const SolveArgs& sa, hs_result* res, double* hist) {
  return dispatch(sa.dtype, opkind_of(sa.A), sa.A->ndim, [&](auto tag) -> hs_status {
    using Tg = decltype(tag);
    using T = typename Tg::T;
    constexpr int OPK = Tg::OPK, NDIM = Tg::NDIM;
    const hs_op* A = sa.A;
    Geom g = geom_of(A);
    Carve c{sa.ws, 0, sa.ws_bytes, true};
    Common cm = carve_common(c, sa.maxit);
    T* r = c.take<T>(g.N);
    T* p0 = c.take<T>(g.N);
    T* p1 = c.take<T>(g.N);
    T* w = c.take<T>(g.N);
    T *D = nullptr, *ax = nullptr, *ay = nullptr, *az = nullptr;
    if (OPK == OP_VARK) {
      D = c.take<T>(g.N);
      ax = c.take<T>(g.N);
      ay = c.take<T>(g.N);
      az = c.take<T>(g.N);
    }
    if (!c.ok) {
      set_error("workspace too small for CG");
      return HS_ERR_WORKSPACE;
    }
    set_last_staging(0);
    if constexpr (std::is_same<T, float>::value && OPK == OP_VARK && NDIM == 3) {
      if (sa.o.staging == 1 && cg32v_eligible(A, sa.o)) {
        // TMA-staged FP32 CG with coefficients formed from k (az holds k in
        // FP32 during the solve; the coefficient arrays are formed afterwards
        // for the true residual)
        const float* k32 = (const float*)A->k;
        if (A->kdt != HS_F32) {
          hs_status s = k_to_f32(A, az, sa.stream);
          if (s != HS_OK) return s;
          k32 = az;
        }
        hs_status s = cg32v_core(A, k32, (const float*)sa.b, (float*)sa.x, sa.tol, sa.maxit, cm, r, p0, p1, w, sa.o,
                                 sa.stream);
        if (s != HS_OK) return s;
        set_last_staging(1);
        if (sa.o.true_residual) {
          s = setup_vark(A, sa.dtype, D, ax, ay, az, false, sa.stream);
          if (s != HS_OK) return s;
        }
        Tail t{A, sa.dtype, D, ax, ay, az, sa.b, sa.x, w};
        return finish_solve(sa, cm, t, res, hist, true);
      }
    }
    if (sa.o.staging == 1) {
      set_error("TMA staging applies to FP32 CG on a 3-D diffusion operator with n_x a multiple of 4, n_x >= 40, "
                "n_y >= 10, n_z >= 3");
      return HS_ERR_INVALID;
    }
    if (OPK == OP_VARK) {
      hs_status s = setup_vark(A, sa.dtype, D, ax, ay, az, false, sa.stream);
      if (s != HS_OK) return s;
    }
    double sigma;
    Coef<T> cf = op_coef<T>(A, D, ax, ay, az, &sigma);
    hs_status s = cg_core<T, OPK, NDIM>(A, cf, sigma, (const T*)sa.b, (T*)sa.x, sa.tol, sa.maxit, cm, r, p0, p1, w,
                                        sa.o, sa.stream);
    if (s != HS_OK) return s;
    Tail t{A, sa.dtype, D, ax, ay, az, sa.b, sa.x, w};
    return finish_solve(sa, cm, t, res, hist, true);
  });
}

// ---- BiCGStab ---------------------------------------------------------------------
// Copies the device restart trace (r_k . r' and a restart flag per iteration)
// into the caller's alpha_trace / restart_iters host arrays.
static hs_status copy_bicgstab_trace(const double* trace, int maxit, int iters, const hs_opts& o, cudaStream_t st) {
  const int n = std::min(std::max(iters, 0), maxit) + 1;
  std::vector<double> h((size_t)2 * n);
  cudaError_t e = cudaMemcpyAsync(h.data(), trace, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "restart trace read-back");
  int q = 0;
  for (int k = 0; k < n; k++) {
    if (o.alpha_trace) o.alpha_trace[k] = h[2 * k];
    if (k > 0 && h[2 * k + 1] != 0.0 && o.restart_iters && q < maxit) o.restart_iters[q++] = k;
  }
  return HS_OK;
}

hs_status run_bicgstab(const SolveArgs& sa, hs_result* res, double* hist) {
  return dispatch(sa.dtype, opkind_of(sa.A), sa.A->ndim, [&](auto tag) -> hs_status {
    using Tg = decltype(tag);
    using T = typename Tg::T;
    constexpr int OPK = Tg::OPK, NDIM = Tg::NDIM;
    const hs_op* A = sa.A;
    Geom g = geom_of(A);
    Carve c{sa.ws, 0, sa.ws_bytes, true};
    Common cm = carve_common(c, sa.maxit);
    T* v[8];
    for (int q = 0; q < 8; q++) v[q] = c.take<T>(g.N);
    T *D = nullptr, *ax = nullptr, *ay = nullptr, *az = nullptr;
    if (OPK == OP_VARK) {
      D = c.take<T>(g.N);
      ax = c.take<T>(g.N);
      ay = c.take<T>(g.N);
      az = c.take<T>(g.N);
    }
    double* trace = c.take<double>(bicgstab_trace_len(sa.maxit));
    if (!c.ok) {
      set_error("workspace too small for BiCGStab");
      return HS_ERR_WORKSPACE;
    }
    const bool want_trace = sa.o.alpha_trace || sa.o.restart_iters;
    if (OPK == OP_VARK) {
      hs_status s = setup_vark(A, sa.dtype, D, ax, ay, az, false, sa.stream);
      if (s != HS_OK) return s;
    }
    double sigma;
    Coef<T> cf = op_coef<T>(A, D, ax, ay, az, &sigma);
    hs_status s = bicgstab_core<T, OPK, NDIM>(A, cf, sigma, (const T*)sa.b, (T*)sa.x, sa.tol, sa.maxit, cm, v, sa.o,
                                              sa.stream, want_trace ? trace : nullptr);
    if (s != HS_OK) return s;
    Tail t{A, sa.dtype, D, ax, ay, az, sa.b, sa.x, v[6]};
    s = finish_solve(sa, cm, t, res, hist, true);
    if (want_trace && s != HS_ERR_CUDA) {
      hs_status s2 = copy_bicgstab_trace(trace, sa.maxit, res->iters, sa.o, sa.stream);
      if (s2 != HS_OK) return s2;
    }
    return s;
  });
}

// ===========================================================================
// Mixed-precision iterative refinement (FP64 outer, FP32 inner).
//   outer, FP64 on the GPU: r = b - A x, ||r|| / ||b|| (stop at tol)
//   inner, FP32:            solve A d = r / ||r|| to inner_tol with CG or
//                           BiCGStab on FP32 vectors and FP32 coefficients,
//                           dot products accumulated in FP64
//   outer, FP64:            x += ||r|| d
// The FP64 and FP32 coefficient arrays of a diffusion operator are formed
// once per solve from the operator's k.
// ===========================================================================

__global__ void k_r_to_f32(const double* __restrict__ r, float* __restrict__ r32, double scale, long long N) {
  for (long long i = gtid(); i < N; i += gstride()) r32[i] = (float)(r[i] * scale);
}
__global__ void k_x_add_f32(double* __restrict__ x, const float* __restrict__ d, double scale, long long N) {
  for (long long i = gtid(); i < N; i += gstride()) x[i] = fma(scale, widen(d[i]), x[i]);
}

struct MixedLayout {
  Common outer;
  double* r64;
  double *D64, *ax64, *ay64, *az64;
  Common inner;
  float* r32;
  float* d32;
  float* v32[8];
  float *D32, *ax32, *ay32, *az32;
};

static MixedLayout carve_mixed(Carve& c, const hs_op* A, const hs_opts& o, int max_outer) {
  MixedLayout L = {};
  const size_t N = (size_t)(A->n[0] * A->n[1] * A->n[2]);
  const bool vark = A->kind == KIND_DIFFUSION;
  const int nvec = (o.inner_solver == HS_SOLVER_BICGSTAB) ? 8 : 4;
  L.outer = carve_common(c, max_outer);
  L.r64 = c.take<double>(N);
  if (vark) {
    L.D64 = c.take<double>(N);
    L.ax64 = c.take<double>(N);
    L.ay64 = c.take<double>(N);
    L.az64 = c.take<double>(N);
  }
  L.inner = carve_common(c, std::max(o.inner_maxit, 1));
  L.r32 = c.take<float>(N);
  L.d32 = c.take<float>(N);
  for (int q = 0; q < nvec; q++) L.v32[q] = c.take<float>(N);
  if (vark) {
    L.D32 = c.take<float>(N);
    L.ax32 = c.take<float>(N);
    L.ay32 = c.take<float>(N);
    L.az32 = c.take<float>(N);
  }
  return L;
}

size_t mixed_ws_bytes(const hs_op* A, const hs_opts& o, int max_outer) {
  Carve c{nullptr, 0, (size_t)-1, true};
  carve_mixed(c, A, o, max_outer);
  return c.off;
}

hs_status run_mixed(const SolveArgs& sa, hs_result* res, double* hist) {
  const hs_op* A = sa.A;
  const Geom g = geom_of(A);
  const int max_outer = sa.maxit;
  Carve c{sa.ws, 0, sa.ws_bytes, true};
  MixedLayout L = carve_mixed(c, A, sa.o, max_outer);
  if (!c.ok) {
    set_error("workspace too small for mixed-precision refinement");
    return HS_ERR_WORKSPACE;
  }
  cudaStream_t st = sa.stream;
  hs_status s;
  // FP32 inner CG on a 3-D diffusion operator with staging 1: the TMA-staged
  // kernel with the face coefficients formed from k (L.D32 then holds k in
  // FP32); otherwise the register-prefetch engine on stored FP32 coefficients
  const bool tma = sa.o.inner_solver != HS_SOLVER_BICGSTAB && sa.o.staging == 1 && cg32v_eligible(A, sa.o);
  if (!tma && sa.o.staging == 1) {
    set_error("TMA staging requested but this problem does not allow it (3-D diffusion, inner CG, n_x a "
              "multiple of 4, n_x >= 40)");
    return HS_ERR_INVALID;
  }
  set_last_staging(tma ? 1 : 0);
  if (A->kind == KIND_DIFFUSION) {
    s = setup_vark(A, HS_F64, L.D64, L.ax64, L.ay64, L.az64, false, st);
    if (s != HS_OK) return s;
    s = tma ? k_to_f32(A, L.D32, st) : setup_vark(A, HS_F32, L.D32, L.ax32, L.ay32, L.az32, false, st);
    if (s != HS_OK) return s;
  }
  const int blocks = (int)std::max<long long>(1, std::min<long long>((g.N + 255) / 256, (long long)sm_count() * 8));
  const bool use_bicg = sa.o.inner_solver == HS_SOLVER_BICGSTAB;
  const int opk = opkind_of(A);
  if (!use_bicg && opk == OP_NONSYM) {
    set_error("mixed precision with inner CG needs a symmetric operator");
    return HS_ERR_INVALID;
  }
  long long inner_total = 0;
  int outer = 0, status = HS_NOT_CONVERGED;
  double rel = -1.0;
  for (;; outer++) {
    // FP64 residual and its norm
    s = residual_norms(A, HS_F64, L.D64, L.ax64, L.ay64, L.az64, sa.b, sa.x, L.r64, &L.outer.ctrl->aux[0],
                       L.outer.partials, st);
    if (s != HS_OK) return s;
    double nrm[2];
    cudaError_t e = cudaMemcpyAsync(nrm, &L.outer.ctrl->aux[0], 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "mixed: residual read-back");
    if (nrm[1] == 0.0) {
      e = cudaMemsetAsync(sa.x, 0, sizeof(double) * (size_t)g.N, st);
      if (e != cudaSuccess) return cuda_fail(e, "mixed: zero x");
      rel = 0.0;
      status = HS_OK;
      if (hist) hist[outer] = 0.0;
      break;
    }
    rel = sqrt(nrm[0] / nrm[1]);
    if (hist && outer <= max_outer) hist[outer] = rel;
    if (!std::isfinite(rel)) {
      status = HS_ERR_NONFINITE;
      break;
    }
    if (rel <= sa.tol) {
      status = HS_OK;
      break;
    }
    if (outer == max_outer) break;
    // FP32 correction solve on the normalised residual.  The step needs the
    // inner residual only down to tol / rel (the FP64 residual after the
    // update is rel times the inner one, plus the FP32 rounding of the
    // correction): a last step close to tol stops its inner solve there
    // (with a factor 2 of margin) instead of running to inner_tol.
    const double itol = sa.o.inner_fixed_tol ? sa.o.inner_tol : inner_tol_for(sa.o.inner_tol, sa.tol, rel);
    const double rn = sqrt(nrm[0]);
    k_r_to_f32<<<blocks, 256, 0, st>>>(L.r64, L.r32, 1.0 / rn, g.N);
    e = cudaMemsetAsync(L.d32, 0, sizeof(float) * (size_t)g.N, st);
    if (e != cudaSuccess) return cuda_fail(e, "mixed: zero correction");
    if (tma)
      s = cg32v_core(A, L.D32, L.r32, L.d32, itol, sa.o.inner_maxit, L.inner, L.v32[0], L.v32[1],
                     L.v32[2], L.v32[3], sa.o, st);
    else
      s = dispatch(HS_F32, opk, A->ndim, [&](auto tag) -> hs_status {
      using Tg = decltype(tag);
      using T = typename Tg::T;
      constexpr int OPK = Tg::OPK, NDIM = Tg::NDIM;
      if constexpr (!std::is_same<T, float>::value) {
        return HS_ERR_INVALID;
      } else {
        double sigma;
        Coef<T> cf = op_coef<T>(A, L.D32, L.ax32, L.ay32, L.az32, &sigma);
        if (use_bicg)
          return bicgstab_core<T, OPK, NDIM>(A, cf, sigma, L.r32, L.d32, itol, sa.o.inner_maxit, L.inner,
                                             L.v32, sa.o, st);
        if constexpr (OPK == OP_NONSYM) {
          return HS_ERR_INVALID;
        } else {
          return cg_core<T, OPK, NDIM>(A, cf, sigma, L.r32, L.d32, itol, sa.o.inner_maxit, L.inner,
                                       L.v32[0], L.v32[1], L.v32[2], L.v32[3], sa.o, st);
        }
      }
    });
    if (s != HS_OK) return s;
    Ctrl h;
    e = cudaMemcpyAsync(&h, L.inner.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "mixed: inner solve");
    inner_total += h.iters;
    if (h.status == DS_TIMEOUT) {
      status = HS_ERR_TIMEOUT;
      break;
    }
    if (h.status == DS_NONFINITE) {
      status = HS_ERR_NONFINITE;
      break;
    }
    // a breakdown or an unconverged inner solve still yields a usable
    // correction; the FP64 residual of the next outer step decides
    k_x_add_f32<<<blocks, 256, 0, st>>>((double*)sa.x, L.d32, rn, g.N);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "mixed: correction update");
  }
  res->iters = outer;
  res->outer = outer;
  res->inner_iters = inner_total;
  res->rel_res = rel;
  res->true_rel_res = rel;
  res->status = status;
  if (status == HS_ERR_NONFINITE) set_error("non-finite value in the refinement");
  if (status == HS_ERR_TIMEOUT) set_error("a device-side wait ran out (timeout)");
  return (hs_status)status;
}

}  // namespace hs
