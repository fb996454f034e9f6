// hs_gs.cu -- exactly lexicographic Gauss-Seidel (section 3.1) on the GPU.
//
// A forward sweep updates idx = i + nx (j + ny k) in ascending order, each
// update reading the entries already updated in the same sweep.  Node
// (i, j, k) depends on the new values at (i-1, j, k), (i, j-1, k), (i, j, k-1)
// and the old ones at (i+1, j, k), (i, j+1, k), (i, j, k+1), so all nodes on a
// hyperplane i + j + k = const are independent.  The kernel applies that
// hyperplane order at two levels, which reproduces the sequential sweep up
// to the rounding order inside a single update (no recolouring):
//
//   * tiles of TX x TY x TZ nodes, tile hyperplane S = I + J + K: tiles on
//     one tile plane are processed in parallel, one grid step per plane;
//     sweep t runs tile plane S = tau - 2t at step tau, so consecutive
//     sweeps of the same direction overlap (sweep t+1 trails sweep t by two
//     tile planes, which leaves every tile's upper neighbours holding the
//     previous sweep's values and its lower neighbours the current sweep's);
//   * inside a tile (staged in shared memory with a one-node halo), one
//     thread per x-line; the line (j, k) processes node i at local step
//     i + j + k.  Lines are dealt to threads in order of j + k so that the
//     32 lines of a warp start within a few steps of each other and the
//     scarce FP64 pipe is not spent on idle lanes.
//
// A backward sweep mirrors every direction.  The symmetric method (forward
// then backward per iteration) runs one sweep per pipeline batch.
#include <math.h>

#include <algorithm>
#include <vector>

#include "hs_internal.h"

namespace hs {

template <int NDIM>
struct GsTile;
// Tile shapes (one thread per x-line: TY * TZ threads per block).  3-D
// default 32 x 8 x 8 (two warps; measured on GB300 at 256^3, 200 sweeps:
// 418 us/sweep against 456 for 32 x 16 x 8, 522 for one-warp 32 x 4 x 8 and
// 32 x 8 x 4, 458-460 for 32 x 4 x 16 and 32 x 16 x 4).  Override at build
// time for measurements (-DHS_GS_TY=.. -DHS_GS_TZ=..).
#ifndef HS_GS_TY
#define HS_GS_TY 8
#endif
#ifndef HS_GS_TZ
#define HS_GS_TZ 8
#endif
template <>
struct GsTile<3> {
  static constexpr int TX = 32, TY = HS_GS_TY, TZ = HS_GS_TZ;
};
template <>
struct GsTile<2> {
  static constexpr int TX = 32, TY = 128, TZ = 1;
};
template <int NDIM>
constexpr int gs_threads() { return GsTile<NDIM>::TY * GsTile<NDIM>::TZ; }

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
  int ntx, nty, ntz, P;
  int maxit;
  int mode;               // HS_GS_FORWARD / BACKWARD / SYMMETRIC
  int check_every;
  double tol;
};

// Line (jl, kl) of thread t when the TY x TZ lines are ordered by jl + kl
// (then kl): the 32 lines of a warp start within a few substeps of each other.
__device__ __forceinline__ void line_of_thread(int t, int TY, int TZ, int& jl, int& kl) {
  int rem = t;
  jl = 0;
  kl = 0;
  for (int dsum = 0; dsum <= TY + TZ - 2; dsum++) {
    const int klo = max(0, dsum - (TY - 1)), khi = min(TZ - 1, dsum);
    const int cnt = khi - klo + 1;
    if (rem < cnt) {
      kl = klo + rem;
      jl = dsum - kl;
      return;
    }
    rem -= cnt;
  }
}

// Relative residual of x through the Jacobi form r_i = a_ii (x'_i - x_i),
// reduced over the grid.  Neighbours come straight from global memory (a
// residual is formed once per check_every sweeps, so no tile staging; this
// also frees the GS block from the tile engine's three-warp minimum).
template <typename T, int OPK, int NDIM>
__device__ bool gs_residual(const GsArgs<T>& a, T* /*sm*/, double* sh, double bb, double* rel) {
  const Geom& g = a.g;
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

// One tile of one sweep: load tile + halo, wavefront in shared memory, store.
template <typename T, int OPK, int NDIM>
__device__ __forceinline__ void gs_tile(const GsArgs<T>& a, T* sm, int tile, bool backward) {
  constexpr int TX = GsTile<NDIM>::TX, TY = GsTile<NDIM>::TY, TZ = GsTile<NDIM>::TZ;
  constexpr int SX = TX + 2, SY = TY + 2, SZ = (NDIM == 3) ? TZ + 2 : 1;
  constexpr int ZOFF = (NDIM == 3) ? 1 : 0;
  const Geom& g = a.g;
  const int I = tile % a.ntx;
  const int J = (tile / a.ntx) % a.nty;
  const int K = tile / (a.ntx * a.nty);
  const int i0 = I * TX, j0 = J * TY, k0 = K * TZ;
  const T* bsrc = (OPK == OP_VARK) ? a.b : a.bD;

  // load tile + one-node halo (zero outside the grid); each thread issues
  // LU independent loads before storing any of them, so a tile costs a few
  // memory round trips instead of one per element
  constexpr int TOT = SX * SY * SZ;
  constexpr int LU = 16;
  constexpr int NT = TY * TZ;
  for (int base = threadIdx.x; base < TOT; base += LU * NT) {
    T v[LU];
#pragma unroll
    for (int u = 0; u < LU; u++) {
      const int e = base + u * NT;
      v[u] = T(0);
      if (e < TOT) {
        const int ii = e % SX, jj = (e / SX) % SY, kk = e / (SX * SY);
        const int gi = i0 + ii - 1, gj = j0 + jj - 1, gk = k0 + kk - ZOFF;
        if (gi >= 0 && gi < g.nx && gj >= 0 && gj < g.ny && gk >= 0 && gk < g.nz)
          v[u] = __ldcg(a.x + (long long)gk * g.plane + (long long)gj * g.nx + gi);
      }
    }
#pragma unroll
    for (int u = 0; u < LU; u++) {
      const int e = base + u * NT;
      if (e < TOT) sm[e] = v[u];
    }
  }
  __syncthreads();

  int jl, kl;
  line_of_thread(threadIdx.x, TY, TZ, jl, kl);
  if (backward) {
    jl = TY - 1 - jl;
    kl = TZ - 1 - kl;
  }
  const int gj = j0 + jl, gk = k0 + kl;
  const bool line_in = (gj < g.ny) && (gk < g.nz);
  const int d = backward ? (TY - 1 - jl) + (TZ - 1 - kl) : jl + kl;
  const int base = ((kl + ZOFF) * SY + (jl + 1)) * SX + 1;
  const long long gbase = (long long)gk * g.plane + (long long)gj * g.nx + i0;
  const int nsteps = TX + TY + TZ - 2;
  // Offsets to the neighbours already updated in this sweep ("new" side:
  // lower neighbours of a forward sweep) and to those not yet updated ("old"
  // side).  The update of a node is split accordingly: the old-side terms
  // are gathered one substep ahead, off the critical path; after the
  // barrier only the new-side terms remain, the x one from a register.
  const int nxo = backward ? 1 : -1;
  const int nyo = backward ? SX : -SX;
  const int nzo = backward ? SX * SY : -SX * SY;
  // local x index of this line at substep s, or -1 when the line is idle
#define HS_IL_AT(S) ((((S) - d) < 0 || ((S) - d) >= TX) ? -1 : \
                     ((line_in && i0 + (backward ? TX - 1 - ((S) - d) : ((S) - d)) < g.nx) ? \
                      (backward ? TX - 1 - ((S) - d) : ((S) - d)) : -1))
  int il = HS_IL_AT(0);
  T yold = T(0), wreg = T(0);
  OpRaw<T, OPK> ocur{};
  if (il >= 0) {
    const int c = base + il;
    const T bv = __ldcg(bsrc + gbase + il);
    ocur = op_fetch<T, OPK, NDIM>(a.cf, g, gbase + il, i0 + il, gj, gk);
    yold = gs_old<T, OPK, NDIM>(a.cf, ocur, bv, sm[c - nxo], sm[c - nyo], NDIM == 3 ? sm[c - nzo] : T(0), backward);
    wreg = sm[c + nxo];
  }
  for (int s = 0; s < nsteps; s++) {
    const int il_n = HS_IL_AT(s + 1);
    T bnext = T(0);
    OpRaw<T, OPK> onext{};
    if (il_n >= 0) {
      bnext = __ldcg(bsrc + gbase + il_n);
      onext = op_fetch<T, OPK, NDIM>(a.cf, g, gbase + il_n, i0 + il_n, gj, gk);
    }
    if (il >= 0) {
      const int c = base + il;
      const T y = gs_new<T, OPK, NDIM>(a.cf, ocur, yold, wreg, sm[c + nyo], NDIM == 3 ? sm[c + nzo] : T(0), backward);
      sm[c] = y;
      wreg = y;
    }
    if (il_n >= 0) {
      // the old-side cells of the next node are written at substep s + 2
      // at the earliest, so they still hold the previous sweep's values
      const int c = base + il_n;
      if (il < 0) wreg = sm[c + nxo];   // first node of the line: x neighbour from the halo
      yold = gs_old<T, OPK, NDIM>(a.cf, onext, bnext, sm[c - nxo], sm[c - nyo], NDIM == 3 ? sm[c - nzo] : T(0),
                                  backward);
    }
    __syncthreads();
    il = il_n;
    ocur = onext;
  }
#undef HS_IL_AT

  // store the tile interior
  for (int e = threadIdx.x; e < TX * TY * TZ; e += blockDim.x) {
    int ii = e % TX, jj = (e / TX) % TY, kk = e / (TX * TY);
    int gi = i0 + ii, gj2 = j0 + jj, gk2 = k0 + kk;
    if (gi < g.nx && gj2 < g.ny && gk2 < g.nz)
      a.x[(long long)gk2 * g.plane + (long long)gj2 * g.nx + gi] = sm[((kk + ZOFF) * SY + (jj + 1)) * SX + ii + 1];
  }
  __syncthreads();
}

// A batch of `nsw` sweeps of one direction, pipelined over tile planes.
template <typename T, int OPK, int NDIM>
__device__ bool gs_batch(const GsArgs<T>& a, T* sm, double* sh, int nsw, bool backward) {
  const int P = a.P;
  const int nsteps = P + 2 * (nsw - 1);
  for (int tau = 0; tau < nsteps; tau++) {
    // active sweeps t with 0 <= tau - 2t < P
    int t_lo = max(0, (tau - P + 2) / 2);
    if (tau - 2 * t_lo >= P) t_lo++;
    int t_hi = min(nsw - 1, tau / 2);
    int total = 0;
    for (int t = t_lo; t <= t_hi; t++) {
      int S = tau - 2 * t;
      int Se = backward ? P - 1 - S : S;
      total += a.plane_off[Se + 1] - a.plane_off[Se];
    }
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
      int rem = item, tile = -1;
      for (int t = t_lo; t <= t_hi; t++) {
        int S = tau - 2 * t;
        int Se = backward ? P - 1 - S : S;
        int cnt = a.plane_off[Se + 1] - a.plane_off[Se];
        if (rem < cnt) {
          tile = a.plane_tiles[a.plane_off[Se] + rem];
          break;
        }
        rem -= cnt;
      }
      if (tile >= 0) gs_tile<T, OPK, NDIM>(a, sm, tile, backward);
    }
    if (!grid_sync(a.cm.ctrl, a.cm.partials, sh)) return false;
  }
  return true;
}

template <typename T, int OPK, int NDIM>
__global__ void __launch_bounds__(gs_threads<NDIM>()) k_gs(GsArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double sh[32 * MAX_SCAL];
  T* sm = reinterpret_cast<T*>(smraw);
  const long long N = a.g.N;

  double acc[1] = {0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    T bv = a.b[i];
    if (OPK != OP_VARK) a.bD[i] = bv * a.invd;
    acc[0] += widen(bv) * widen(bv);
  }
  block_sum<1>(acc, sh);
  double bb[1];
  if (!grid_reduce<1>(a.cm.ctrl, a.cm.partials, acc, bb, sh)) return;
  if (bb[0] == 0.0) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
      a.x[i] = T(0);
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
    if (!gs_residual<T, OPK, NDIM>(a, sm, sh, bb[0], &rel)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.cm.hist[0] = rel;
    if (!(rel > a.tol)) status = isfinite(rel) ? DS_CONVERGED : DS_NONFINITE;
    else status = DS_MAXIT;
  }
  if (!(a.tol > 0.0) || status == DS_MAXIT) {
    while (done < a.maxit) {
      int nb = (a.tol > 0.0) ? min(a.check_every, a.maxit - done) : a.maxit - done;
      if (a.mode == HS_GS_SYMMETRIC) {
        for (int q = 0; q < nb; q++) {
          if (!gs_batch<T, OPK, NDIM>(a, sm, sh, 1, false)) return;
          if (!gs_batch<T, OPK, NDIM>(a, sm, sh, 1, true)) return;
        }
      } else {
        if (!gs_batch<T, OPK, NDIM>(a, sm, sh, nb, a.mode == HS_GS_BACKWARD)) return;
      }
      done += nb;
      if (a.tol > 0.0) {
        if (!gs_residual<T, OPK, NDIM>(a, sm, sh, bb[0], &rel)) return;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
          for (int q = done - nb + 1; q < done; q++) a.cm.hist[q] = nan("");  // not evaluated
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

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

template <int NDIM>
static void tile_counts(const hs_op* A, int* ntx, int* nty, int* ntz) {
  *ntx = (int)((A->n[0] + GsTile<NDIM>::TX - 1) / GsTile<NDIM>::TX);
  *nty = (int)((A->n[1] + GsTile<NDIM>::TY - 1) / GsTile<NDIM>::TY);
  *ntz = (int)((A->n[2] + GsTile<NDIM>::TZ - 1) / GsTile<NDIM>::TZ);
}

static void gs_counts(const hs_op* A, int* ntiles, int* P) {
  int a, b, c;
  if (A->ndim >= 3) tile_counts<3>(A, &a, &b, &c);
  else tile_counts<2>(A, &a, &b, &c);
  *ntiles = a * b * c;
  *P = a + b + c - 2;
}

size_t gs_ws_vectors(const hs_op* A, hs_dtype dt) {
  size_t N = (size_t)(A->n[0] * A->n[1] * A->n[2]);
  size_t es = dt == HS_F64 ? 8 : 4;
  // 27-point sweep: b / a_ii and one progress word per block (hs_gs27.cu)
  if (opkind_of(A) == OP_BOX27) return ((N * es + 255) & ~(size_t)255) + gs27_progress_bytes();
  int nt, P;
  gs_counts(A, &nt, &P);
  size_t ints = (size_t)nt + P + 1;
  return ((N * es + 255) & ~(size_t)255) + ((ints * 4 + 255) & ~(size_t)255);
}

template <typename T>
static Coef<T> gs_jacobi_coef(const hs_op* A, T* invd, double* d2) {
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

template <typename T, int OPK, int NDIM>
static hs_status gs_run_t(const SolveArgs& sa, hs_result* res, double* hist) {
  constexpr int TX = GsTile<NDIM>::TX, TY = GsTile<NDIM>::TY, TZ = GsTile<NDIM>::TZ;
  constexpr int THREADS = TY * TZ;
  static_assert(THREADS % 32 == 0 && THREADS <= 1024, "GS tiles use whole warps of lines");
  const hs_op* A = sa.A;
  Geom g = geom_of(A);
  Carve c{sa.ws, 0, sa.ws_bytes, true};
  Common cm = carve_common(c, sa.maxit);
  GsArgs<T> a = {};
  a.bD = c.take<T>(g.N);
  int ntx, nty, ntz;
  tile_counts<NDIM>(A, &ntx, &nty, &ntz);
  if (NDIM == 2) ntz = 1;
  const int ntiles = ntx * nty * ntz, P = ntx + nty + ntz - 2;
  int* tabs = c.take<int>((size_t)ntiles + P + 1);
  T *D = nullptr, *ax = nullptr, *ay = nullptr, *az = nullptr;
  if (OPK == OP_VARK) {
    D = c.take<T>(g.N);
    ax = c.take<T>(g.N);
    ay = c.take<T>(g.N);
    az = c.take<T>(g.N);
  }
  if (!c.ok) {
    set_error("workspace too small for Gauss-Seidel");
    return HS_ERR_WORKSPACE;
  }
  // tile planes: offsets then tile ids grouped by I + J + K
  std::vector<int> host((size_t)ntiles + P + 1);
  {
    std::vector<int> cnt(P + 1, 0);
    for (int t = 0; t < ntiles; t++) {
      int I = t % ntx, J = (t / ntx) % nty, K = t / (ntx * nty);
      cnt[I + J + K + 1]++;
    }
    for (int s = 0; s < P; s++) cnt[s + 1] += cnt[s];
    for (int s = 0; s <= P; s++) host[s] = cnt[s];
    std::vector<int> fill(cnt.begin(), cnt.end() - 1);
    for (int t = 0; t < ntiles; t++) {
      int I = t % ntx, J = (t / ntx) % nty, K = t / (ntx * nty);
      host[P + 1 + fill[I + J + K]++] = t;
    }
  }
  cudaError_t e = cudaMemcpyAsync(tabs, host.data(), host.size() * sizeof(int), cudaMemcpyHostToDevice, sa.stream);
  if (e != cudaSuccess) return cuda_fail(e, "tile table upload");
  {
    double t = sa.o.timeout_s > 0 ? sa.o.timeout_s : 2.0;
    Ctrl h = {};
    h.timeout_ns = (unsigned long long)(t * 1e9);
    h.rel_res = -1.0;
    e = cudaMemcpyAsync(cm.ctrl, &h, sizeof(Ctrl), cudaMemcpyHostToDevice, sa.stream);
    if (e != cudaSuccess) return cuda_fail(e, "control init");
    e = cudaStreamSynchronize(sa.stream);  // host staging buffers go out of scope below
    if (e != cudaSuccess) return cuda_fail(e, "control init");
  }
  if (OPK == OP_VARK) {
    hs_status s = setup_vark(A, sa.dtype, D, ax, ay, az, true, sa.stream);
    if (s != HS_OK) return s;
    a.cf.D = D;
    a.cf.ax = ax;
    a.cf.ay = ay;
    a.cf.az = az;
    a.dscale2 = 1.0;
  } else {
    a.cf = gs_jacobi_coef<T>(A, &a.invd, &a.dscale2);
  }
  a.g = g;
  a.b = (const T*)sa.b;
  a.x = (T*)sa.x;
  a.cm = cm;
  a.plane_off = tabs;
  a.plane_tiles = tabs + P + 1;
  a.ntx = ntx;
  a.nty = nty;
  a.ntz = ntz;
  a.P = P;
  a.maxit = sa.maxit;
  a.mode = sa.o.gs_mode;
  a.check_every = sa.o.check_every;
  a.tol = sa.tol;
  const int sx = TX + 2, sy = TY + 2, sz = (NDIM == 3) ? TZ + 2 : 1;
  const size_t smem = (size_t)sx * sy * sz * sizeof(T);
  auto kern = k_gs<T, OPK, NDIM>;
  // static shared memory (reduction scratch) comes on top of the dynamic
  // tile, so always raise the dynamic limit to what the tile needs
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "shared-memory attribute");
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, smem);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
  if (per_sm < 1) {
    set_error("Gauss-Seidel kernel cannot be resident");
    return HS_ERR_CUDA;
  }
  int grid = std::min(per_sm * sm_count(), MAX_BLOCKS);
  void* args[] = {&a};
  e = cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(THREADS), args, smem, sa.stream);
  if (e != cudaSuccess) return cuda_fail(e, "cooperative launch");
  if (OPK == OP_VARK && sa.o.true_residual) {
    hs_status s = setup_vark(A, sa.dtype, D, ax, ay, az, false, sa.stream);
    if (s != HS_OK) return s;
  }
  return finish_solve_pub(sa, cm, D, ax, ay, az, a.bD, res, hist, sa.tol > 0.0);
}

hs_status run_gauss_seidel(const SolveArgs& sa, hs_result* res, double* hist) {
  const int opk = opkind_of(sa.A);
  const bool d3 = sa.A->ndim >= 3;
  if (opk == OP_BOX27) return run_gauss_seidel27(sa, res, hist);
#define HS_GS(TT, OK)                                                        \
  if (opk == OK) return d3 ? gs_run_t<TT, OK, 3>(sa, res, hist) : gs_run_t<TT, OK, 2>(sa, res, hist);
  if (sa.dtype == HS_F64) {
    HS_GS(double, OP_SYM)
    HS_GS(double, OP_NONSYM)
    HS_GS(double, OP_VARK)
  } else {
    HS_GS(float, OP_SYM)
    HS_GS(float, OP_NONSYM)
    HS_GS(float, OP_VARK)
  }
#undef HS_GS
  set_error("unsupported operator");
  return HS_ERR_INVALID;
}

}  // namespace hs
