// hs_gs27.cu -- exactly lexicographic Gauss-Seidel for the 27-point HPCG
// operator (section 3.1 with the system of section 4.1).
//
// A forward sweep updates node (i, j, k) after its 13 lower neighbours (all
// box neighbours of smaller index).  They all lie on smaller values of
// h = i + 2j + 4k and the 13 upper neighbours on larger ones, so the nodes of
// one hyperplane h are independent and the sweep is the sequence of
// hyperplanes h = 0 .. H-1, H = (nx-1) + 2(ny-1) + 4(nz-1) + 1; a backward
// sweep runs them in the reverse order.  Unlike the 7-point case there is no
// tile order (a lower neighbour such as (i+1, j-1, k) can lie in the next
// tile along x while that tile needs this one's values), so every hyperplane
// is one grid-wide step and nodes are updated in place in global memory.
//
// Consecutive sweeps of one direction are pipelined: sweep t runs hyperplane
// tau - 8t at step tau.  A node's neighbours lie within 7 hyperplanes, so the
// upper neighbours sweep t+1 reads hold sweep t's values and no two active
// hyperplanes of a step touch each other's nodes.
//
// Hyperplane h holds, for each k with a non-empty range, the lines j with
// 0 <= h - 4k - 2j < nx; threads take (k, slot) pairs with M = nx/2 + 1
// slots per k (the longest j range).
#include <algorithm>
#include <cmath>

#include "hs_krylov.cuh"

namespace hs {

template <typename T>
struct Gs27Args {
  Geom g;
  T g27;            // 1 / 27 (Jacobi-form coupling of every neighbour)
  T invd;           // 1 / 27
  double dscale2;   // 27^2 (residual = a_ii (x' - x))
  const T* b;
  T* bD;            // b / 27
  T* x;
  Common cm;
  int H;            // hyperplanes per sweep
  int M;            // slots per k
  int maxit;
  int mode;         // HS_GS_FORWARD / BACKWARD / SYMMETRIC
  int check_every;
  double tol;
};

constexpr int GS27_LAG = 8;

// k range of hyperplane h (empty when klo > khi).
__device__ __forceinline__ void gs27_krange(const Geom& g, int h, int& klo, int& khi) {
  khi = min(g.nz - 1, h / 4);
  const int r = h - (g.nx - 1) - 2 * (g.ny - 1);   // 4k >= r
  klo = r <= 0 ? 0 : (r + 3) / 4;
}

// x_i <- (b_i + sum of the 26 neighbours) / 27, in place.
template <typename T>
__device__ __forceinline__ void gs27_node(const Gs27Args<T>& a, int i, int j, int k) {
  const Geom& g = a.g;
  const long long idx = (long long)k * g.plane + (long long)j * g.nx + i;
  T box = T(0);
#pragma unroll
  for (int dz = -1; dz <= 1; dz++)
#pragma unroll
    for (int dy = -1; dy <= 1; dy++)
#pragma unroll
      for (int dx = -1; dx <= 1; dx++) {
        const int ii = i + dx, jj = j + dy, kk = k + dz;
        if (ii >= 0 && ii < g.nx && jj >= 0 && jj < g.ny && kk >= 0 && kk < g.nz)
          box += __ldcg(a.x + idx + (long long)dz * g.plane + (long long)dy * g.nx + dx);
      }
  const T c = __ldcg(a.x + idx);
  a.x[idx] = fma(a.g27, box - c, __ldcg(a.bD + idx));
}

// Nodes of hyperplane h handed out over the whole grid.
template <typename T>
__device__ __forceinline__ void gs27_plane(const Gs27Args<T>& a, int h) {
  const Geom& g = a.g;
  int klo, khi;
  gs27_krange(g, h, klo, khi);
  if (klo > khi) return;
  const long long slots = (long long)(khi - klo + 1) * a.M;
  for (long long e = gtid(); e < slots; e += gstride()) {
    const int k = klo + (int)(e / a.M);
    const int q = (int)(e % a.M);
    const int rem = h - 4 * k;                       // = i + 2j
    const int jlo = rem - (g.nx - 1) <= 0 ? 0 : (rem - (g.nx - 1) + 1) / 2;
    const int j = jlo + q;
    if (j >= g.ny || 2 * j > rem) continue;
    gs27_node(a, rem - 2 * j, j, k);
  }
}

// nsw pipelined sweeps of one direction.
template <typename T>
__device__ bool gs27_batch(const Gs27Args<T>& a, double* sh, int nsw, bool backward) {
  const int H = a.H;
  const int nsteps = H + GS27_LAG * (nsw - 1);
  for (int tau = 0; tau < nsteps; tau++) {
    const int t_hi = min(nsw - 1, tau / GS27_LAG);
    for (int t = t_hi; t >= 0; t--) {
      const int s = tau - GS27_LAG * t;
      if (s >= H) break;   // older sweeps have finished
      gs27_plane(a, backward ? H - 1 - s : s);
    }
    if (!grid_sync(a.cm.ctrl, a.cm.partials, sh)) return false;
  }
  return true;
}

// Relative residual through the Jacobi form, reduced over the grid.
template <typename T>
__device__ bool gs27_residual(const Gs27Args<T>& a, double* sh, double bb, double* rel) {
  const Geom& g = a.g;
  double acc[1] = {0.0};
  for (long long idx = gtid(); idx < g.N; idx += gstride()) {
    const int i = (int)(idx % g.nx);
    const int j = (int)((idx / g.nx) % g.ny);
    const int k = (int)(idx / g.plane);
    T box = T(0);
    for (int dz = -1; dz <= 1; dz++)
      for (int dy = -1; dy <= 1; dy++)
        for (int dx = -1; dx <= 1; dx++) {
          const int ii = i + dx, jj = j + dy, kk = k + dz;
          if (ii >= 0 && ii < g.nx && jj >= 0 && jj < g.ny && kk >= 0 && kk < g.nz)
            box += __ldcg(a.x + idx + (long long)dz * g.plane + (long long)dy * g.nx + dx);
        }
    const T c = __ldcg(a.x + idx);
    const T d = fma(a.g27, box - c, __ldcg(a.bD + idx)) - c;
    acc[0] += widen(d) * widen(d);
  }
  block_sum<1>(acc, sh);
  double rr[1];
  if (!grid_reduce<1>(a.cm.ctrl, a.cm.partials, acc, rr, sh)) return false;
  *rel = sqrt(rr[0] * a.dscale2 / bb);
  return true;
}

template <typename T>
__global__ void __launch_bounds__(256) k_gs27(Gs27Args<T> a) {
  __shared__ double sh[32 * MAX_SCAL];
  const long long N = a.g.N;
  double acc[1] = {0.0};
  for (long long i = gtid(); i < N; i += gstride()) {
    const T bv = a.b[i];
    a.bD[i] = bv * a.invd;
    acc[0] += widen(bv) * widen(bv);
  }
  block_sum<1>(acc, sh);
  double bb[1];
  if (!grid_reduce<1>(a.cm.ctrl, a.cm.partials, acc, bb, sh)) return;
  if (bb[0] == 0.0) {
    for (long long i = gtid(); i < N; i += gstride()) a.x[i] = T(0);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.cm.hist[0] = 0.0;
      a.cm.ctrl->iters = 0;
      a.cm.ctrl->rel_res = 0.0;
      atomicCAS(&a.cm.ctrl->status, 0, (int)DS_CONVERGED);
    }
    return;
  }
  int done = 0, status = DS_CONVERGED;
  double rel = -1.0;
  if (a.tol > 0.0) {
    if (!gs27_residual(a, sh, bb[0], &rel)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.cm.hist[0] = rel;
    status = !(rel > a.tol) ? (isfinite(rel) ? DS_CONVERGED : DS_NONFINITE) : DS_MAXIT;
  }
  if (!(a.tol > 0.0) || status == DS_MAXIT) {
    while (done < a.maxit) {
      const int nb = (a.tol > 0.0) ? min(a.check_every, a.maxit - done) : a.maxit - done;
      if (a.mode == HS_GS_SYMMETRIC) {
        for (int q = 0; q < nb; q++) {
          if (!gs27_batch(a, sh, 1, false)) return;
          if (!gs27_batch(a, sh, 1, true)) return;
        }
      } else {
        if (!gs27_batch(a, sh, nb, a.mode == HS_GS_BACKWARD)) return;
      }
      done += nb;
      if (a.tol > 0.0) {
        if (!gs27_residual(a, sh, bb[0], &rel)) return;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
          for (int q = done - nb + 1; q < done; q++) a.cm.hist[q] = nan("");   // not evaluated
          a.cm.hist[done] = rel;
        }
        if (!isfinite(rel)) {
          status = DS_NONFINITE;
          break;
        }
        if (rel <= a.tol) {
          status = DS_CONVERGED;
          break;
        }
        status = DS_MAXIT;
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.cm.ctrl->iters = done;
    a.cm.ctrl->rel_res = rel;
    atomicCAS(&a.cm.ctrl->status, 0, status);
  }
}

template <typename T>
static hs_status gs27_t(const SolveArgs& sa, hs_result* res, double* hist) {
  const hs_op* A = sa.A;
  const Geom g = geom_of(A);
  Carve c{sa.ws, 0, sa.ws_bytes, true};
  Common cm = carve_common(c, sa.maxit);
  Gs27Args<T> a = {};
  a.bD = c.take<T>(g.N);
  if (!c.ok) {
    set_error("workspace too small for Gauss-Seidel");
    return HS_ERR_WORKSPACE;
  }
  hs_status s = init_ctrl(cm, sa.o, sa.stream);
  if (s != HS_OK) return s;
  a.g = g;
  a.g27 = (T)(1.0 / 27.0);
  a.invd = (T)(1.0 / 27.0);
  a.dscale2 = 27.0 * 27.0;
  a.b = (const T*)sa.b;
  a.x = (T*)sa.x;
  a.cm = cm;
  a.H = (g.nx - 1) + 2 * (g.ny - 1) + 4 * (g.nz - 1) + 1;
  a.M = g.nx / 2 + 1;
  a.maxit = sa.maxit;
  a.mode = sa.o.gs_mode;
  a.check_every = sa.o.check_every;
  a.tol = sa.tol;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gs27<T>, 256, 0);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
  if (per_sm < 1) {
    set_error("Gauss-Seidel kernel cannot be resident");
    return HS_ERR_CUDA;
  }
  int grid = std::min(per_sm * sm_count(), MAX_BLOCKS);
  if (sa.o.max_blocks > 0) grid = std::min(grid, sa.o.max_blocks);
  void* args[] = {&a};
  s = launch_coop((const void*)k_gs27<T>, grid, 256, args, 0, sa.stream);
  if (s != HS_OK) return s;
  return finish_solve_pub(sa, cm, nullptr, nullptr, nullptr, nullptr, a.bD, res, hist, sa.tol > 0.0);
}

hs_status run_gauss_seidel27(const SolveArgs& sa, hs_result* res, double* hist) {
  return sa.dtype == HS_F64 ? gs27_t<double>(sa, res, hist) : gs27_t<float>(sa, res, hist);
}

}  // namespace hs
