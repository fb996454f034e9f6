// hs_cgnb.cu -- CG-NB, the paper's nonblocking conjugate gradient (section 3.2,
// Algorithm 1), as a persistent kernel with ONE reduce-barrier per iteration.
//
// Algorithm 1 applies the SpMV to r_j instead of p_j and obtains A p_j by the
// recurrence q_j = A p_j = w_j + beta_j q_j-1 with w_j = A r_j, so that the
// reduction of alpha_n,j = r_j.r_j can overlap the SpMV.  On the GPU the
// iteration's second reduction, alpha_d,j = q_j.p_j, is merged into the first
// by expanding it over the vectors one pass sees before beta_j is known:
//   q_j.p_j = (w_j + beta_j q_j-1).(r_j + beta_j p_j-1)
//           = r_j.w_j + 2 beta_j r_j.q_j-1 + beta_j^2 q_j-1.p_j-1
// (w_j.p_j-1 = r_j.A p_j-1 = r_j.q_j-1 for symmetric A; q_j-1.p_j-1 is the
// previous alpha_d).  The three terms come from the vectors themselves, with
// no appeal to the orthogonality of r_j to p_j-1 that holds only in exact
// arithmetic (the shorter form r_j.w_j - beta_j alpha_n,j / alpha_j-1 relies
// on it and converged measurably later than Algorithm 1 on coefficient-
// contrast problems), so one pass computes everything an iteration needs and
// one barrier ends it:
//
//   source, every node the stencil reads (halo included):
//     q_k = w_k + beta_k q_k-1,  r_k+1 = r_k - alpha_k q_k   (stored if owned)
//   sink, owned nodes:
//     w_k+1 = A r_k+1,  p_k = r_k + beta_k p_k-1,  x_k+1 = x_k + alpha_k p_k,
//     partial sums r_k+1.r_k+1, r_k+1.w_k+1 and r_k+1.q_k (q_k formed again
//     from w_k and q_k-1, bitwise as the source formed it)
//
// r, w and q are ping-ponged (a tile reads its neighbours' old values while
// they write new ones); p and x are updated in place (owned nodes only).
// Everything runs on the scaled operator S = A / sigma (see op_coef): w = S r,
// q = S p, and alpha below multiplies q (the true step length is alpha/sigma).
#include <algorithm>
#include <cmath>

#include "hs_krylov.cuh"

namespace hs {

template <typename T>
struct CgnbArgs {
  Geom g;
  Tiling tl;
  Coef<T> cf;
  double sigma;
  const T* b;
  T* x;
  T* r[2];
  T* w[2];
  T* q[2];
  T* p;
  Common cm;
  int maxit;
  double tol;
  int paper_order;
};

// q_k = w_k + beta q_k-1 ; r_k+1 = r_k - alpha q_k ; stencil input r_k+1.
template <typename T>
struct CgnbSrc {
  const T* w;
  const T* qold;
  const T* rold;
  T* qnew;
  T* rnew;
  T alpha, beta;
  struct Raw {
    T w, q, r;
  };
  __device__ __forceinline__ Raw fetch(long long idx) const {
    return Raw{__ldcg(w + idx), __ldcg(qold + idx), __ldcg(rold + idx)};
  }
  __device__ __forceinline__ T make(const Raw& v, long long idx, bool own) const {
    const T qn = fma(beta, v.q, v.w);
    const T rn = fma(-alpha, qn, v.r);
    if (own) {
      qnew[idx] = qn;
      rnew[idx] = rn;
    }
    return rn;
  }
};

// w_k+1 = S r_k+1 ; p_k = r_k + beta p_k-1 ; x += (alpha / sigma) p_k ;
// r.r, r.w, r.q_k.
template <typename T, int OPK, int NDIM>
struct CgnbSink {
  static constexpr bool kBox = OPK == OP_BOX27;
  Coef<T> cf;
  Geom g;
  T* wnew;
  const T* rold;
  const T* wk;      // w_k and q_k-1: q_k = w_k + beta q_k-1
  const T* qkm1;
  T* p;
  T* x;
  T beta, ax;
  double acc[3];
  struct Raw {
    OpRaw<T, OPK> o;
    T r, p, x, w, q;
  };
  __device__ __forceinline__ Raw fetch(long long idx, int i, int j, int k) const {
    return Raw{op_fetch<T, OPK, NDIM>(cf, g, idx, i, j, k), __ldcg(rold + idx), __ldcg(p + idx), __ldcg(x + idx),
               __ldcg(wk + idx), __ldcg(qkm1 + idx)};
  }
  __device__ __forceinline__ void operator()(long long idx, const Nbr<T>& nb, const Raw& q, int, int, int) {
    const T wv = op_apply<T, OPK, NDIM>(cf, q.o, nb);
    wnew[idx] = wv;
    const T pv = fma(beta, q.p, q.r);
    p[idx] = pv;
    x[idx] = fma(ax, pv, q.x);
    const T qk = fma(beta, q.q, q.w);
    const double rc = widen(nb.c);
    acc[0] += rc * rc;
    acc[1] += rc * widen(wv);
    acc[2] += rc * widen(qk);
  }
};

// w = S r and r.w (start-up pass).
template <typename T, int OPK, int NDIM>
struct CgnbStartSink {
  static constexpr bool kBox = OPK == OP_BOX27;
  Coef<T> cf;
  Geom g;
  T* w;
  double acc[1];
  using Raw = OpRaw<T, OPK>;
  __device__ __forceinline__ Raw fetch(long long idx, int i, int j, int k) const {
    return op_fetch<T, OPK, NDIM>(cf, g, idx, i, j, k);
  }
  __device__ __forceinline__ void operator()(long long idx, const Nbr<T>& nb, const Raw& o, int, int, int) {
    const T wv = op_apply<T, OPK, NDIM>(cf, o, nb);
    w[idx] = wv;
    acc[0] += widen(nb.c) * widen(wv);
  }
};

template <typename T, int OPK, int NDIM>
__global__ void __launch_bounds__(512) k_cg_nb(CgnbArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double sh[32 * MAX_SCAL];
  T* sm = reinterpret_cast<T*>(smraw);
  const Team tm = grid_team(a.cm.ctrl, a.cm.partials);
  const long long N = a.g.N;
  const long long st = tm.stride();
  const T sig = (T)a.sigma;
  // p_-1 = q_-1 = 0: the first iteration's recurrences then start from r_0, w_0
  for (long long i = tm.tid(); i < N; i += st) {
    a.p[i] = T(0);
    a.q[1][i] = T(0);
  }
  // r_0 = b - A x_0 ; ||r_0||^2 ; ||b||^2
  ResidualSink<T, OPK, NDIM> rsink{a.cf, a.g, sig, a.b, a.r[0], {0.0, 0.0}};
  {
    LoadSrc<T, true> src{a.x};
    for (int item = tm.rank; item < a.tl.items(); item += tm.size)
      zmarch_item<T, NDIM, 1>(a.g, a.tl, item, sm, src, rsink);
  }
  block_sum<2>(rsink.acc, sh);
  double s2[2];
  if (!team_reduce<2>(tm, rsink.acc, s2, sh)) return;
  double an = s2[0];
  const double bb = s2[1];
  if (bb == 0.0) {
    for (long long i = tm.tid(); i < N; i += st) a.x[i] = T(0);
    if (tm.lead()) a.cm.hist[0] = 0.0;
    team_finish(tm, DS_CONVERGED, 0, 0.0);
    return;
  }
  double rel = sqrt(an / bb);
  if (tm.lead()) a.cm.hist[0] = rel;
  if (rel <= a.tol || a.maxit == 0) {
    team_finish(tm, rel <= a.tol ? DS_CONVERGED : DS_MAXIT, 0, rel);
    return;
  }
  // w_0 = S r_0 ; delta_0 = r_0.w_0 = alpha_d,0 (beta_0 = 0)
  double d0[1];
  {
    CgnbStartSink<T, OPK, NDIM> sink{a.cf, a.g, a.w[0], {0.0}};
    LoadSrc<T, true> src{a.r[0]};
    for (int item = tm.rank; item < a.tl.items(); item += tm.size)
      zmarch_item<T, NDIM, 1>(a.g, a.tl, item, sm, src, sink);
    block_sum<1>(sink.acc, sh);
    if (!team_reduce<1>(tm, sink.acc, d0, sh)) return;
  }
  if (!(d0[0] > 0.0) || !isfinite(d0[0])) {
    team_finish(tm, isfinite(d0[0]) ? DS_BREAKDOWN : DS_NONFINITE, 0, rel);
    return;
  }
  double alpha = an / d0[0], beta = 0.0, ad_prev = d0[0];
  int it = 0, status = DS_MAXIT, cur = 0;
  while (it < a.maxit) {
    // ---- the iteration's single pass (buffers: cur = k, 1 - cur = k + 1 / k - 1)
    CgnbSrc<T> src{a.w[cur], a.q[1 - cur], a.r[cur], a.q[cur], a.r[1 - cur], (T)alpha, (T)beta};
    CgnbSink<T, OPK, NDIM> sink{a.cf,    a.g,        a.w[1 - cur], a.r[cur], a.w[cur], a.q[1 - cur],
                                a.p,     a.x,        (T)beta,      (T)(alpha / a.sigma), {0.0, 0.0, 0.0}};
    for (int item = tm.rank; item < a.tl.items(); item += tm.size)
      zmarch_item<T, NDIM, 1>(a.g, a.tl, item, sm, src, sink);
    block_sum<3>(sink.acc, sh);
    double rw[3];
    if (!team_reduce<3>(tm, sink.acc, rw, sh)) return;
    it++;
    cur = 1 - cur;
    const double an_new = rw[0];
    rel = sqrt(an_new / bb);
    if (tm.lead()) a.cm.hist[it] = rel;
    if (!isfinite(rel) || !isfinite(rw[1])) {
      status = DS_NONFINITE;
      break;
    }
    const double beta_new = an_new / an;
    const double ad = rw[1] + beta_new * (2.0 * rw[2] + beta_new * ad_prev);   // q.p expanded
    if (rel <= a.tol) {
      status = DS_CONVERGED;
      if (a.paper_order) {
        // Algorithm 1's order tests at the top of the next iteration and then
        // applies x = x_l + alpha_l p_l: p_l = r_l + beta_l p_l-1, one more step
        if (!(ad > 0.0)) break;
        const T tb = (T)beta_new, tax = (T)(an_new / ad / a.sigma);
        for (long long i = tm.tid(); i < N; i += st) {
          const T pv = fma(tb, ldcg(a.p + i), ldcg(a.r[cur] + i));
          a.x[i] = fma(tax, pv, ldcg(a.x + i));
        }
      }
      break;
    }
    if (!(ad > 0.0)) {
      status = DS_BREAKDOWN;
      break;
    }
    beta = beta_new;
    alpha = an_new / ad;
    an = an_new;
    ad_prev = ad;
  }
  team_finish(tm, status, it, rel);
}

template <typename T, int OPK, int NDIM>
static hs_status cg_nb_t(const SolveArgs& sa, hs_result* res, double* hist) {
  const hs_op* A = sa.A;
  const Geom g = geom_of(A);
  Carve c{sa.ws, 0, sa.ws_bytes, true};
  Common cm = carve_common(c, sa.maxit);
  CgnbArgs<T> a = {};
  for (int q = 0; q < 2; q++) {
    a.r[q] = c.take<T>(g.N);
    a.w[q] = c.take<T>(g.N);
    a.q[q] = c.take<T>(g.N);
  }
  a.p = c.take<T>(g.N);
  T *D = nullptr, *ax = nullptr, *ay = nullptr, *az = nullptr;
  if (OPK == OP_VARK) {
    D = c.take<T>(g.N);
    ax = c.take<T>(g.N);
    ay = c.take<T>(g.N);
    az = c.take<T>(g.N);
  }
  if (!c.ok) {
    set_error("workspace too small for CG-NB");
    return HS_ERR_WORKSPACE;
  }
  hs_status s = init_ctrl(cm, sa.o, sa.stream);
  if (s != HS_OK) return s;
  if (OPK == OP_VARK) {
    s = setup_vark(A, sa.dtype, D, ax, ay, az, false, sa.stream);
    if (s != HS_OK) return s;
  }
  a.g = g;
  a.cf = op_coef<T>(A, D, ax, ay, az, &a.sigma);
  a.b = (const T*)sa.b;
  a.x = (T*)sa.x;
  a.cm = cm;
  a.maxit = sa.maxit;
  a.tol = sa.tol;
  a.paper_order = sa.o.paper_order;
  const int by = rows_for(g, sa.o);
  const size_t smem = slab_bytes<T>(by, 1);
  int grid = 0;
  s = plan_persistent(k_cg_nb<T, OPK, NDIM>, 32 * by, smem, g, by, true, &grid, &a.tl, sa.o, 1);
  if (s != HS_OK) return s;
  void* args[] = {&a};
  s = launch_coop((const void*)k_cg_nb<T, OPK, NDIM>, grid, 32 * by, args, smem, sa.stream);
  if (s != HS_OK) return s;
  s = hs_dbg_take(sa.stream);
  if (s != HS_OK) return s;
  return finish_solve_pub(sa, cm, D, ax, ay, az, a.w[0], res, hist, true);
}

hs_status run_cg_nb(const SolveArgs& sa, hs_result* res, double* hist) {
  const int opk = opkind_of(sa.A);
  const bool d3 = sa.A->ndim >= 3;
#define HS_NB(TT, OK) \
  if (opk == OK) return d3 ? cg_nb_t<TT, OK, 3>(sa, res, hist) : cg_nb_t<TT, OK, 2>(sa, res, hist);
  if (sa.dtype == HS_F64) {
    HS_NB(double, OP_SYM)
    HS_NB(double, OP_VARK)
    if (opk == OP_BOX27) return cg_nb_t<double, OP_BOX27, 3>(sa, res, hist);
  } else {
    HS_NB(float, OP_SYM)
    HS_NB(float, OP_VARK)
    if (opk == OP_BOX27) return cg_nb_t<float, OP_BOX27, 3>(sa, res, hist);
  }
#undef HS_NB
  set_error("CG-NB needs a symmetric operator");
  return HS_ERR_INVALID;
}

}  // namespace hs
