// hs_krylov.cuh -- device code of the fused Krylov solvers (CG, BiCGStab) and
// the host helpers that set up their operator coefficients.  Shared by the
// standalone solver kernels (hs_kernels.cu) and the batched solver
// (hs_batch.cu), which run the same iteration bodies on teams of blocks.
#pragma once
#include <math.h>

#include "hs_internal.h"

namespace hs {

// Columns per lane of the tile engine for each kernel family (see
// hs_stencil.cuh).  Measured on GB300: two columns per lane neither speeds up
// the FP64-pipe-bound solver passes nor helps the HBM-bound FP32 ones (whose
// occupancy drops with the extra registers), so the solvers use one; the
// single-pass SpMV / residual kernels use two.
constexpr int CX_ST = 2;    // SpMV / residual (7-point operators)
template <int OPK>
__host__ __device__ constexpr int cx_st() { return OPK == OP_BOX27 ? 1 : CX_ST; }
constexpr int CX_BI = 1;    // BiCGStab
// FP32 Jacobi: two columns per lane (measured at 256^3: 91 -> 64 us/sweep;
// the FP32 sweep is memory-latency bound and gains from the second chain).
#ifndef HS_JAC_CX32
#define HS_JAC_CX32 2
#endif
template <typename T, int OPK>
__host__ __device__ constexpr int cx_jac() {
  return (sizeof(T) == 4 && OPK != OP_BOX27) ? HS_JAC_CX32 : 1;
}
template <typename T, int OPK>
__host__ __device__ constexpr int cx_cg() { return 1; }

// Global index / stride helpers for grid-stride element loops.
__device__ __forceinline__ long long gtid() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ long long gstride() { return (long long)gridDim.x * blockDim.x; }

template <typename T>
__device__ __forceinline__ T ldcg(const T* p) {
  return __ldcg(p);
}

__device__ __forceinline__ bool finite_d(double v) { return isfinite(v); }

// Writes the final solver outcome (block 0, thread 0 only).
__device__ __forceinline__ void finish(Ctrl* c, int status, int iters, double rel) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c->iters = iters;
    c->rel_res = rel;
    atomicCAS(&c->status, 0, status);
  }
}

// Outcome of an iteration body, identical in every block of the team (all
// blocks take their decisions from the same reduced scalars).  ok = false:
// a team barrier was abandoned (timeout or an error status already posted),
// the body returned early and the control block holds the status.
struct BodyOut {
  int status;
  int iters;
  double rel;
  int restarts;
  bool ok;
};

// Writes the final solver outcome of a team (its lead thread only).
__device__ __forceinline__ void team_finish(const Team& tm, int status, int iters, double rel) {
  if (tm.lead()) {
    tm.ctrl->iters = iters;
    tm.ctrl->rel_res = rel;
    atomicCAS(&tm.ctrl->status, 0, status);
  }
}
__device__ __forceinline__ void team_finish(const Team& tm, const BodyOut& o) {
  if (!o.ok) return;
  if (tm.lead()) tm.ctrl->restarts = o.restarts;
  team_finish(tm, o.status, o.iters, o.rel);
}

// ===========================================================================
// Common sinks
// ===========================================================================

// y = A x (scaled operator times sigma).
template <typename T, int OPK, int NDIM>
struct SpmvSink {
  static constexpr bool kBox = OPK == OP_BOX27;
  Coef<T> cf;
  Geom g;
  T sigma;
  T* y;
  using Raw = OpRaw<T, OPK>;
  __device__ __forceinline__ Raw fetch(long long idx, int i, int j, int k) const {
    return op_fetch<T, OPK, NDIM>(cf, g, idx, i, j, k);
  }
  __device__ __forceinline__ void operator()(long long idx, const Nbr<T>& nb, const Raw& o, int, int, int) {
    T v = op_apply<T, OPK, NDIM>(cf, o, nb);
    if (OPK != OP_VARK) v *= sigma;
    y[idx] = v;
  }
};

// r = b - A x, accumulating ||r||^2 and ||b||^2.
template <typename T, int OPK, int NDIM>
struct ResidualSink {
  static constexpr bool kBox = OPK == OP_BOX27;
  Coef<T> cf;
  Geom g;
  T sigma;
  const T* b;
  T* r;
  double acc[2];
  struct Raw {
    OpRaw<T, OPK> o;
    T b;
  };
  __device__ __forceinline__ Raw fetch(long long idx, int i, int j, int k) const {
    return Raw{op_fetch<T, OPK, NDIM>(cf, g, idx, i, j, k), __ldg(b + idx)};
  }
  __device__ __forceinline__ void operator()(long long idx, const Nbr<T>& nb, const Raw& q, int, int, int) {
    T v = op_apply<T, OPK, NDIM>(cf, q.o, nb);
    T rv = (OPK == OP_VARK) ? q.b - v : fma(-sigma, v, q.b);
    r[idx] = rv;
    acc[0] += widen(rv) * widen(rv);
    acc[1] += widen(q.b) * widen(q.b);
  }
};

// Elementwise passes process ILP elements per thread per round: all loads of
// a round are issued before any arithmetic or store, so several memory
// requests are in flight per thread.  The element -> thread assignment and
// the per-thread accumulation order are fixed by the launch shape.
constexpr int ILP = 4;

// ===========================================================================
// CG: classical Hestenes-Stiefel (section 3.2) in two fused passes.
//   pass 1 (stencil):  p = r + beta p_old (on the fly, halo included),
//                      w = A p / sigma, partial p.w
//   pass 2 (elements): x += alpha p, r -= alpha A p, partial r.r
// p is double-buffered so that halo reads of p_old never race with stores.
// ===========================================================================

template <typename T>
struct CgArgs {
  Geom g;
  Tiling tl;
  Coef<T> cf;
  double sigma;   // A = sigma * (scaled operator)
  const T* b;
  T* x;
  T* r;
  T* p0;
  T* p1;
  T* w;
  Common cm;
  int maxit;
  double tol;
};

// p = r + beta p_old (or p = r), stored for owned nodes.
template <typename T>
struct PUpdateSrc {
  const T* r;
  const T* pold;
  T* pnew;
  T beta;
  bool first;
  struct Raw {
    T r, p;
  };
  __device__ __forceinline__ Raw fetch(long long idx) const {
    Raw q;
    q.r = __ldcg(r + idx);
    q.p = first ? T(0) : __ldcg(pold + idx);
    return q;
  }
  __device__ __forceinline__ T make(const Raw& q, long long idx, bool own) const {
    T pv = first ? q.r : fma(beta, q.p, q.r);
    if (own) pnew[idx] = pv;
    return pv;
  }
};

// w = A p / sigma, accumulating p.w.  With XUPD the node's x also takes the
// previous iteration's step, x += alpha_prev p_prev: the x update rides on
// this FP64-pipe-bound pass instead of lengthening the memory-bound
// elementwise pass.
template <typename T, int OPK, int NDIM, bool XUPD>
struct ApDotSink {
  static constexpr bool kBox = OPK == OP_BOX27;
  Coef<T> cf;
  Geom g;
  T* w;
  T* x;
  const T* pold;
  T ax;
  double acc[1];
  using Raw = OpRaw<T, OPK>;
  __device__ __forceinline__ Raw fetch(long long idx, int i, int j, int k) const {
    return op_fetch<T, OPK, NDIM>(cf, g, idx, i, j, k);
  }
  __device__ __forceinline__ void operator()(long long idx, const Nbr<T>& nb, const Raw& o, int, int, int) {
    T wv = op_apply<T, OPK, NDIM>(cf, o, nb);
    w[idx] = wv;
    acc[0] += widen(nb.c) * widen(wv);
    // p_old was read two planes earlier by the source: an L2 hit; not
    // prefetched, which would raise the register count of every pass
    if constexpr (XUPD) x[idx] = fma(ax, __ldcg(pold + idx), __ldcg(x + idx));
  }
};

// The CG iteration run by one team of blocks (the whole grid for a standalone
// solve, a subset of blocks in the batched solver).
// XDEFER: the x update of iteration k runs in pass 1 of iteration k+1
// (ApDotSink<XUPD>), leaving pass 2 with r alone.  It pays where pass 1 is
// FP64-pipe bound (standalone FP64); FP32 passes are memory bound and the
// batched kernel is register bound, so they keep x in pass 2.
template <typename T, int OPK, int NDIM, int CX = cx_cg<T, OPK>(), bool XDEFER = false>
__device__ BodyOut cg_body(const CgArgs<T>& a, const Team& tm, T* sm, double* sh) {
  const long long N = a.g.N;
  const T sig = (T)a.sigma;

  // r = b - A x ; ||r||^2, ||b||^2
  ResidualSink<T, OPK, NDIM> rsink{a.cf, a.g, sig, a.b, a.r, {0.0, 0.0}};
  {
    LoadSrc<T, true> src{a.x};
    for (int item = tm.rank; item < a.tl.items(); item += tm.size)
      zmarch_item<T, NDIM, CX>(a.g, a.tl, item, sm, src, rsink);
  }
  block_sum<2>(rsink.acc, sh);
  double s2[2];
  if (!team_reduce<2>(tm, rsink.acc, s2, sh)) return BodyOut{DS_TIMEOUT, 0, -1.0, 0, false};
  double rr = s2[0];
  const double bb = s2[1];
  if (bb == 0.0) {
    for (long long i = tm.tid(); i < N; i += tm.stride()) a.x[i] = T(0);
    if (tm.lead() && a.cm.hist) a.cm.hist[0] = 0.0;
    return BodyOut{DS_CONVERGED, 0, 0.0, 0, true};
  }
  double rel = sqrt(rr / bb);
  if (tm.lead() && a.cm.hist) a.cm.hist[0] = rel;
  if (rel <= a.tol || a.maxit == 0) {
    return BodyOut{rel <= a.tol ? DS_CONVERGED : DS_MAXIT, 0, rel, 0, true};
  }

  double beta = 0.0, alpha_prev = 0.0;
  bool first = true;
  int it = 0, status = DS_MAXIT;
  const long long st = tm.stride();
  while (it < a.maxit) {
    it++;
    const T* pold = (it & 1) ? a.p0 : a.p1;
    T* pnew = (it & 1) ? a.p1 : a.p0;
    // ---- pass 1: p = r + beta p_old ; w = A p / sigma ; p.w ; x += alpha_prev p_old
    PUpdateSrc<T> src{a.r, pold, pnew, (T)beta, first};
    double pw[1], acc0[1];
    {
      // first iteration: no step pending; x += 0 * r (r is finite, p_old
      // undefined) leaves x unchanged
      ApDotSink<T, OPK, NDIM, XDEFER> sink{a.cf, a.g, a.w, a.x, first ? a.r : pold,
                                           first ? T(0) : (T)(alpha_prev / a.sigma), {0.0}};
      for (int item = tm.rank; item < a.tl.items(); item += tm.size)
        zmarch_item<T, NDIM, CX>(a.g, a.tl, item, sm, src, sink);
      acc0[0] = sink.acc[0];
    }
    block_sum<1>(acc0, sh);
    if (!team_reduce<1>(tm, acc0, pw, sh)) return BodyOut{DS_TIMEOUT, it, rel, 0, false};
    if (!(pw[0] > 0.0) || !finite_d(pw[0])) {
      status = finite_d(pw[0]) ? DS_BREAKDOWN : DS_NONFINITE;
      return BodyOut{status, it, rel, 0, true};   // x holds x_{it-1} in both forms
    }
    const double ar = rr / pw[0];           // multiplies w = A p / sigma
    const T tar = (T)ar;
    double acc1[1] = {0.0};
    if constexpr (XDEFER) {
      // ---- pass 2: r -= alpha A p ; r.r   (x follows in the next pass 1)
      long long i = tm.tid();
      for (; i + (ILP - 1) * st < N; i += ILP * st) {
        T wv[ILP], rv[ILP];
#pragma unroll
        for (int u = 0; u < ILP; u++) {
          const long long q = i + u * st;
          wv[u] = ldcg(a.w + q);
          rv[u] = ldcg(a.r + q);
        }
#pragma unroll
        for (int u = 0; u < ILP; u++) {
          const long long q = i + u * st;
          rv[u] = fma(-tar, wv[u], rv[u]);
          a.r[q] = rv[u];
          acc1[0] += widen(rv[u]) * widen(rv[u]);
        }
      }
      for (; i < N; i += st) {
        T rv = fma(-tar, ldcg(a.w + i), ldcg(a.r + i));
        a.r[i] = rv;
        acc1[0] += widen(rv) * widen(rv);
      }
    } else {
      // ---- pass 2: x += alpha p ; r -= alpha A p ; r.r
      const T tax = (T)(ar / a.sigma);      // multiplies p
      long long i = tm.tid();
      for (; i + (ILP - 1) * st < N; i += ILP * st) {
        T pv[ILP], wv[ILP], xv[ILP], rv[ILP];
#pragma unroll
        for (int u = 0; u < ILP; u++) {
          const long long q = i + u * st;
          pv[u] = ldcg(pnew + q);
          wv[u] = ldcg(a.w + q);
          xv[u] = ldcg(a.x + q);
          rv[u] = ldcg(a.r + q);
        }
#pragma unroll
        for (int u = 0; u < ILP; u++) {
          const long long q = i + u * st;
          xv[u] = fma(tax, pv[u], xv[u]);
          rv[u] = fma(-tar, wv[u], rv[u]);
          a.x[q] = xv[u];
          a.r[q] = rv[u];
          acc1[0] += widen(rv[u]) * widen(rv[u]);
        }
      }
      for (; i < N; i += st) {
        T xv = fma(tax, ldcg(pnew + i), ldcg(a.x + i));
        T rv = fma(-tar, ldcg(a.w + i), ldcg(a.r + i));
        a.x[i] = xv;
        a.r[i] = rv;
        acc1[0] += widen(rv) * widen(rv);
      }
    }
    block_sum<1>(acc1, sh);
    double rn[1];
    if (!team_reduce<1>(tm, acc1, rn, sh)) return BodyOut{DS_TIMEOUT, it, rel, 0, false};
    alpha_prev = ar;
    rel = sqrt(rn[0] / bb);
    if (tm.lead() && a.cm.hist) a.cm.hist[it] = rel;
    if (!finite_d(rel)) {
      status = DS_NONFINITE;
      break;
    }
    if (rel <= a.tol) {
      status = DS_CONVERGED;
      break;
    }
    beta = rn[0] / rr;
    rr = rn[0];
    first = false;
  }
  // the last step of x, x += alpha p (same element -> thread map as the
  // callers' elementwise passes, so no barrier is needed before they read x)
  if constexpr (XDEFER) {
    const T* plast = (it & 1) ? a.p1 : a.p0;
    const T tax = (T)(alpha_prev / a.sigma);
    for (long long i = tm.tid(); i < N; i += st) a.x[i] = fma(tax, ldcg(plast + i), ldcg(a.x + i));
  }
  return BodyOut{status, it, rel, 0, true};
}

// ===========================================================================
// BiCGStab with Algorithm 2's normalised shadow residual and restart rule,
// three fused passes per iteration:
//   pass 1 (stencil):  p = r + beta (p_old - omega v_old) (or p = r after a
//                      start/restart, which also stores r' = r/||r||),
//                      v = A p / sigma, partial v.r'
//   pass 2 (stencil):  s = r - alpha A p (on the fly), t = A s / sigma,
//                      partials s.s, t.s, t.t
//   pass 3 (elements): x += alpha p + omega s, r = s - omega A s,
//                      partials r.r', r.r
// ===========================================================================

template <typename T>
struct BiArgs {
  Geom g;
  Tiling tl;
  Coef<T> cf;
  double sigma;
  const T* b;
  T* x;
  T* r;
  T* rs;
  T* p0;
  T* p1;
  T* v0;
  T* v1;
  T* s;
  T* t;
  Common cm;
  int maxit;
  double tol;
  double reps;
  int paper_order;   // Algorithm 2's statement order (BiCGStab-B1)
  double* trace;     // optional, 2 (maxit + 1) doubles: per iteration k, r_k . r'
                     // and 1.0 if a restart followed (entry 0: r_0 . r')
};

// p = r + beta (p_old - omega sigma v_old), or p = r on (re)start.  The
// restart case is a separate instantiation (RESTART): a run-time flag would
// let the compiler predicate the other branch's FP64 work, which still issues.
template <typename T, bool RESTART>
struct BiPSrc {
  const T* r;
  const T* pold;
  const T* vold;
  T* pnew;
  T beta, ws;
  struct Raw {
    T r, p, v;
  };
  __device__ __forceinline__ Raw fetch(long long idx) const {
    Raw q;
    q.r = __ldcg(r + idx);
    if constexpr (RESTART) {
      q.p = T(0);
      q.v = T(0);
    } else {
      q.p = __ldcg(pold + idx);
      q.v = __ldcg(vold + idx);
    }
    return q;
  }
  __device__ __forceinline__ T make(const Raw& q, long long idx, bool own) const {
    T pv;
    if constexpr (RESTART)
      pv = q.r;
    else
      pv = fma(beta, fma(-ws, q.v, q.p), q.r);
    if (own) pnew[idx] = pv;
    return pv;
  }
};

// v = A p / sigma; r' = r/||r|| stored on (re)start; partial v.r'.
template <typename T, int OPK, int NDIM, bool RESTART>
struct BiVSink {
  static constexpr bool kBox = OPK == OP_BOX27;
  Coef<T> cf;
  Geom g;
  const T* r;
  T* rs;
  T* vnew;
  T inv_rn;
  double acc[1];
  struct Raw {
    OpRaw<T, OPK> o;
    T q;   // r (restart) or r'
  };
  __device__ __forceinline__ Raw fetch(long long idx, int i, int j, int k) const {
    return Raw{op_fetch<T, OPK, NDIM>(cf, g, idx, i, j, k), RESTART ? __ldcg(r + idx) : __ldcg(rs + idx)};
  }
  __device__ __forceinline__ void operator()(long long idx, const Nbr<T>& nb, const Raw& q, int, int, int) {
    T vv = op_apply<T, OPK, NDIM>(cf, q.o, nb);
    vnew[idx] = vv;
    T rsv = q.q;
    if constexpr (RESTART) {
      rsv = q.q * inv_rn;
      rs[idx] = rsv;
    }
    acc[0] += widen(vv) * widen(rsv);
  }
};

// s = r - alpha sigma v, stored for owned nodes.
template <typename T>
struct BiSSrc {
  const T* r;
  const T* v;
  T* s;
  T as;
  struct Raw {
    T r, v;
  };
  __device__ __forceinline__ Raw fetch(long long idx) const { return Raw{__ldcg(r + idx), __ldcg(v + idx)}; }
  __device__ __forceinline__ T make(const Raw& q, long long idx, bool own) const {
    T sv = fma(-as, q.v, q.r);
    if (own) s[idx] = sv;
    return sv;
  }
};

// t = A s / sigma; partials s.s, t.s, t.t.
template <typename T, int OPK, int NDIM>
struct BiTSink {
  static constexpr bool kBox = OPK == OP_BOX27;
  Coef<T> cf;
  Geom g;
  T* t;
  double acc[3];
  using Raw = OpRaw<T, OPK>;
  __device__ __forceinline__ Raw fetch(long long idx, int i, int j, int k) const {
    return op_fetch<T, OPK, NDIM>(cf, g, idx, i, j, k);
  }
  __device__ __forceinline__ void operator()(long long idx, const Nbr<T>& nb, const Raw& o, int, int, int) {
    T tv = op_apply<T, OPK, NDIM>(cf, o, nb);
    t[idx] = tv;
    const double sv = widen(nb.c), td = widen(tv);
    acc[0] += sv * sv;
    acc[1] += td * sv;
    acc[2] += td * td;
  }
};

// The BiCGStab iteration run by one team of blocks.
template <typename T, int OPK, int NDIM, int CX = CX_BI>
__device__ BodyOut bicgstab_body(const BiArgs<T>& a, const Team& tm, T* sm, double* sh) {
  const long long N = a.g.N;
  const T sig = (T)a.sigma;

  ResidualSink<T, OPK, NDIM> rsink{a.cf, a.g, sig, a.b, a.r, {0.0, 0.0}};
  {
    LoadSrc<T, true> src{a.x};
    for (int item = tm.rank; item < a.tl.items(); item += tm.size)
      zmarch_item<T, NDIM, CX>(a.g, a.tl, item, sm, src, rsink);
  }
  block_sum<2>(rsink.acc, sh);
  double s2[2];
  if (!team_reduce<2>(tm, rsink.acc, s2, sh)) return BodyOut{DS_TIMEOUT, 0, -1.0, 0, false};
  double brr = s2[0];
  const double bb = s2[1];
  if (bb == 0.0) {
    for (long long i = tm.tid(); i < N; i += tm.stride()) a.x[i] = T(0);
    if (tm.lead() && a.cm.hist) a.cm.hist[0] = 0.0;
    return BodyOut{DS_CONVERGED, 0, 0.0, 0, true};
  }
  double rel = sqrt(brr / bb);
  if (tm.lead() && a.cm.hist) a.cm.hist[0] = rel;
  if (rel <= a.tol || a.maxit == 0) {
    return BodyOut{rel <= a.tol ? DS_CONVERGED : DS_MAXIT, 0, rel, 0, true};
  }

  double alpha_n = sqrt(brr);   // r . r' with r' = r / ||r||
  double inv_rn = 1.0 / sqrt(brr);
  if (tm.lead() && a.trace) {
    a.trace[0] = alpha_n;
    a.trace[1] = 0.0;
  }
  bool restart = true;          // p = r and r' = r/||r|| in the next pass 1
  double beta = 0.0, omega = 0.0;
  int it = 0, status = DS_MAXIT, restarts = 0;
  const long long st = tm.stride();
  while (it < a.maxit) {
    it++;
    const T* pold = (it & 1) ? a.p0 : a.p1;
    T* pnew = (it & 1) ? a.p1 : a.p0;
    const T* vold = (it & 1) ? a.v0 : a.v1;
    T* vnew = (it & 1) ? a.v1 : a.v0;
    // ---- pass 1
    double ad[1];
    {
      double acc1[1];
      if (restart) {
        BiPSrc<T, true> src{a.r, pold, vold, pnew, (T)beta, (T)(omega * a.sigma)};
        BiVSink<T, OPK, NDIM, true> sink{a.cf, a.g, a.r, a.rs, vnew, (T)inv_rn, {0.0}};
        for (int item = tm.rank; item < a.tl.items(); item += tm.size)
          zmarch_item<T, NDIM, CX>(a.g, a.tl, item, sm, src, sink);
        acc1[0] = sink.acc[0];
      } else {
        BiPSrc<T, false> src{a.r, pold, vold, pnew, (T)beta, (T)(omega * a.sigma)};
        BiVSink<T, OPK, NDIM, false> sink{a.cf, a.g, a.r, a.rs, vnew, (T)inv_rn, {0.0}};
        for (int item = tm.rank; item < a.tl.items(); item += tm.size)
          zmarch_item<T, NDIM, CX>(a.g, a.tl, item, sm, src, sink);
        acc1[0] = sink.acc[0];
      }
      block_sum<1>(acc1, sh);
      if (!team_reduce<1>(tm, acc1, ad, sh)) return BodyOut{DS_TIMEOUT, it, rel, restarts, false};
    }
    const double alpha_d = a.sigma * ad[0];
    if (alpha_d == 0.0 || !finite_d(alpha_d)) {
      status = finite_d(alpha_d) ? DS_BREAKDOWN : DS_NONFINITE;
      break;
    }
    const double alpha = alpha_n / alpha_d;
    // ---- pass 2
    double st3[3];
    {
      BiSSrc<T> src{a.r, vnew, a.s, (T)(alpha * a.sigma)};
      BiTSink<T, OPK, NDIM> sink{a.cf, a.g, a.t, {0.0, 0.0, 0.0}};
      for (int item = tm.rank; item < a.tl.items(); item += tm.size)
        zmarch_item<T, NDIM, CX>(a.g, a.tl, item, sm, src, sink);
      block_sum<3>(sink.acc, sh);
      if (!team_reduce<3>(tm, sink.acc, st3, sh)) return BodyOut{DS_TIMEOUT, it, rel, restarts, false};
    }
    const double srel = sqrt(st3[0] / bb);
    if (!a.paper_order && srel <= a.tol) {
      const T ta = (T)alpha;
      for (long long i = tm.tid(); i < N; i += st) a.x[i] = fma(ta, ldcg(pnew + i), ldcg(a.x + i));
      if (tm.lead() && a.cm.hist) a.cm.hist[it] = srel;
      rel = srel;
      status = DS_CONVERGED;
      break;
    }
    const double ts = a.sigma * st3[1], tt = a.sigma * a.sigma * st3[2];
    if (tt == 0.0 || !finite_d(tt) || !finite_d(ts)) {
      status = finite_d(tt) && finite_d(ts) ? DS_BREAKDOWN : DS_NONFINITE;
      break;
    }
    omega = ts / tt;
    if (omega == 0.0) {
      status = DS_BREAKDOWN;
      break;
    }
    const T ta = (T)alpha, tom = (T)omega, toms = (T)(omega * a.sigma);
    if (a.paper_order && rel <= a.tol) {
      // Algorithm 2's order: the test on the residual of x_j comes after
      // omega_j, and the loop ends with x = x_j + alpha_j p_j + omega_j s_j
      for (long long i = tm.tid(); i < N; i += st)
        a.x[i] = fma(tom, ldcg(a.s + i), fma(ta, ldcg(pnew + i), ldcg(a.x + i)));
      if (tm.lead() && a.cm.hist) a.cm.hist[it] = nan("");   // residual of the last step not formed
      status = DS_CONVERGED;
      break;
    }
    // ---- pass 3
    double acc4[2] = {0.0, 0.0};
    long long i = tm.tid();
    for (; i + (ILP - 1) * st < N; i += ILP * st) {
      T sv[ILP], pv[ILP], xv[ILP], tv[ILP], rsv[ILP];
#pragma unroll
      for (int u = 0; u < ILP; u++) {
        const long long q = i + u * st;
        sv[u] = ldcg(a.s + q);
        pv[u] = ldcg(pnew + q);
        xv[u] = ldcg(a.x + q);
        tv[u] = ldcg(a.t + q);
        rsv[u] = ldcg(a.rs + q);
      }
#pragma unroll
      for (int u = 0; u < ILP; u++) {
        const long long q = i + u * st;
        T xn = fma(tom, sv[u], fma(ta, pv[u], xv[u]));
        T rn = fma(-toms, tv[u], sv[u]);
        a.x[q] = xn;
        a.r[q] = rn;
        acc4[0] += widen(rn) * widen(rsv[u]);
        acc4[1] += widen(rn) * widen(rn);
      }
    }
    for (; i < N; i += st) {
      const long long q = i;
      T sv = ldcg(a.s + q);
      T xn = fma(tom, sv, fma(ta, ldcg(pnew + q), ldcg(a.x + q)));
      T rn = fma(-toms, ldcg(a.t + q), sv);
      a.x[q] = xn;
      a.r[q] = rn;
      acc4[0] += widen(rn) * widen(ldcg(a.rs + q));
      acc4[1] += widen(rn) * widen(rn);
    }
    block_sum<2>(acc4, sh);
    double rn2[2];
    if (!team_reduce<2>(tm, acc4, rn2, sh)) return BodyOut{DS_TIMEOUT, it, rel, restarts, false};
    rel = sqrt(rn2[1] / bb);
    if (tm.lead() && a.cm.hist) a.cm.hist[it] = rel;
    if (tm.lead() && a.trace) {
      a.trace[2 * it] = rn2[0];
      a.trace[2 * it + 1] = 0.0;
    }
    if (!finite_d(rel) || !finite_d(rn2[0])) {
      status = DS_NONFINITE;
      break;
    }
    if (!a.paper_order && rel <= a.tol) {
      status = DS_CONVERGED;
      break;
    }
    if (a.reps > 0.0 && sqrt(fabs(rn2[0])) < a.reps) {
      restart = true;
      alpha_n = sqrt(rn2[1]);
      inv_rn = 1.0 / sqrt(rn2[1]);
      restarts++;
    } else {
      restart = false;
      beta = rn2[0] / (alpha_d * omega);
      alpha_n = rn2[0];
    }
    if (tm.lead() && a.trace && restart) a.trace[2 * it + 1] = 1.0;
  }
  return BodyOut{status, it, rel, restarts, true};
}

// ---------------------------------------------------------------------------
// Host helpers
// ---------------------------------------------------------------------------

// Scaled coefficients: divide by sigma = -xu so that xu becomes exactly -1.
template <typename T>
inline Coef<T> scaled_coef(const hs_op* A, double* sigma) {
  Coef<T> cf = {};
  ConstRow c = const_row(A);
  double s = -c.xu;
  *sigma = s;
  cf.d = (T)(c.d / s);
  cf.xl = (T)(c.xl / s);
  cf.xu = (T)(-1.0);
  cf.yl = (T)(c.yl / s);
  cf.yu = (T)(c.yu / s);
  cf.zl = (T)(c.zl / s);
  cf.zu = (T)(c.zu / s);
  // 27-point: A x = 27 x - (box - x) = 28 x - box (s = 1)
  if (A->kind == KIND_HPCG27) cf.d = (T)(c.d + 1.0);
  return cf;
}

inline int rows_per_tile(const Geom& g) {
  // 2-D grids are small: more, shorter tiles; 3-D: 8 rows (256 threads).
  if (g.nz == 1) return g.ny >= 64 ? 8 : 4;
  return 8;
}

// Rows per tile: the caller's choice (hs_opts.tile_rows, 4 to 16) or the
// heuristic above.
inline int rows_for(const Geom& g, const hs_opts& o) {
  if (o.tile_rows >= 4 && o.tile_rows <= 16) return o.tile_rows;
  return rows_per_tile(g);
}

template <typename T>
inline size_t slab_bytes(int by, int cx) {
  return (size_t)2 * (by + 2) * (BX * cx + 2) * sizeof(T);
}

// Operator coefficients for stencil kernels (scaled form, or var-k arrays).
template <typename T>
inline Coef<T> op_coef(const hs_op* A, const void* D, const void* ax, const void* ay, const void* az,
                       double* sigma) {
  if (A->kind == KIND_DIFFUSION) {
    Coef<T> cf = {};
    cf.D = (const T*)D;
    cf.ax = (const T*)ax;
    cf.ay = (const T*)ay;
    cf.az = (const T*)az;
    *sigma = 1.0;
    return cf;
  }
  return scaled_coef<T>(A, sigma);
}

// ---- persistent launch planning ------------------------------------------------
template <typename K>
inline hs_status plan_persistent(K kernel, int block, size_t smem, const Geom& g, int by, bool src_expensive,
                                 int* grid_out, Tiling* tl_out, const hs_opts& o, int cx) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
  if (per_sm < 1) {
    set_error("persistent kernel cannot be resident (block %d, smem %zu)", block, smem);
    return HS_ERR_CUDA;
  }
  int grid = std::min(per_sm * sm_count(), MAX_BLOCKS);
  if (o.max_blocks > 0) grid = std::min(grid, o.max_blocks);
  Tiling tl = choose_tiling(g, by, grid, src_expensive, o.tile_planes, cx);
  grid = std::max(1, std::min(grid, tl.items()));
  *tl_out = choose_tiling(g, by, grid, src_expensive, o.tile_planes, cx);
  *grid_out = grid;
  return HS_OK;
}


}  // namespace hs
