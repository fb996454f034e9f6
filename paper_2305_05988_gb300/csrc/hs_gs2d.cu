// hs_gs2d.cu -- exactly lexicographic Gauss-Seidel (section 3.1) on small
// 2-D (and 1-D) grids held on chip.
//
// One block holds the whole iterate in shared
// memory and sweeps it along anti-diagonals i + j = d, the node order of the
// tile kernel's intra-tile wavefront applied to the entire grid.  Sweeps of
// one direction are pipelined: sweep t works on diagonal s - 2t at step s, so
// the old-side neighbours of its nodes (diagonal d + 1) still hold sweep
// t - 1's values and the new-side ones (diagonal d - 1) already hold sweep
// t's; nodes handled in one step lie on diagonals two apart and never
// neighbour each other, so one block barrier per step orders everything.  A
// batch of n sweeps takes n_x + n_y - 1 + 2 (n - 1) steps instead of the
// n (n_x + n_y - 1) tile-plane steps of the multi-block schedule, with no
// grid-wide wait.  Thread (i, q) owns column i and the sweeps t = q (mod Q).
// The update arithmetic is that of the tile schedule (gs_old then gs_new,
// hs_gs.cuh), so the iterates are bitwise those of the other schedules.
//
// The cluster form (k_gs2dc, below) splits the rows over the CTAs of one
// thread-block cluster.
#include <cooperative_groups.h>

#include "hs_gs.cuh"

namespace hs {

template <typename T, int OPK>
__device__ __forceinline__ void gs2d_node(const GsArgs<T>& a, T* xs, T bv, int i, int j, bool bw) {
  const Geom& g = a.g;
  const int nx = g.nx, ny = g.ny;
  const int c = j * nx + i;
  if (!HS_IN_BOUNDS(c, g.N)) return;
  const T vW = i > 0 ? xs[c - 1] : T(0);
  const T vE = i + 1 < nx ? xs[c + 1] : T(0);
  const T vS = j > 0 ? xs[c - nx] : T(0);
  const T vN = j + 1 < ny ? xs[c + nx] : T(0);
  const OpRaw<T, OPK> o = op_fetch<T, OPK, 2>(a.cf, g, c, i, j, 0);
  // old side: upper neighbours of a forward sweep, lower ones of a backward
  const T yold = gs_old<T, OPK, 2>(a.cf, o, bv, bw ? vW : vE, bw ? vS : vN, T(0), bw);
  xs[c] = gs_new<T, OPK, 2>(a.cf, o, yold, bw ? vE : vW, bw ? vN : vS, T(0), bw);
}

// nsw sweeps of one direction, pipelined two diagonals apart.  (Loading the
// right-hand sides one step ahead measured slower: the index arithmetic it
// adds outweighs the L2 latency it hides.)
template <typename T, int OPK>
__device__ void gs2d_batch(const GsArgs<T>& a, T* xs, const T* bsrc, int nsw, bool bw) {
  const int nx = a.g.nx, ny = a.g.ny;
  const int Q = blockDim.x / nx;                 // sweep lanes per column
  const int i = threadIdx.x % nx, q = threadIdx.x / nx;
  const bool active = q < Q;
  const int dmax = nx + ny - 2;
  const int nsteps = dmax + 1 + 2 * (nsw - 1);
  const int ii = bw ? nx - 1 - i : i;             // the column in the sweep's frame
  for (int s = 0; s < nsteps; s++) {
    if (active) {
      // sweeps t with a node in column i at this step: row s - 2t - i of the
      // sweep's own frame lies in [0, ny), i.e. t in [t_lo, t_hi]; this
      // thread takes those with t = q (mod Q)
      const int t_lo = max(0, (s - i - (ny - 1) + 1) >> 1);
      const int t_hi = min(nsw - 1, (s - i) >> 1);
      for (int t = t_lo + (((q - t_lo) % Q) + Q) % Q; t <= t_hi; t += Q) {
        const int r = s - 2 * t - i;
        const int jj = bw ? ny - 1 - r : r;
        if (HS_IN_BOUNDS(jj * nx + ii, a.g.N)) gs2d_node<T, OPK>(a, xs, __ldcg(bsrc + jj * nx + ii), ii, jj, bw);
      }
    }
    __syncthreads();
  }
}

// Relative residual ||b - A x|| / ||b|| of the iterate in shared memory,
// through the Jacobi form as gs_residual.
template <typename T, int OPK>
__device__ double gs2d_residual(const GsArgs<T>& a, const T* xs, const T* bsrc, double* sh, double bb) {
  const Geom& g = a.g;
  double acc[1] = {0.0};
  for (int c = threadIdx.x; c < (int)g.N; c += blockDim.x) {
    const int i = c % g.nx, j = c / g.nx;
    Nbr<T> nb;
    nb.c = xs[c];
    nb.w = i > 0 ? xs[c - 1] : T(0);
    nb.e = i + 1 < g.nx ? xs[c + 1] : T(0);
    nb.s = j > 0 ? xs[c - g.nx] : T(0);
    nb.n = j + 1 < g.ny ? xs[c + g.nx] : T(0);
    nb.b = nb.t = T(0);
    const OpRaw<T, OPK> o = op_fetch<T, OPK, 2>(a.cf, g, c, i, j, 0);
    T d = jacobi_apply<T, OPK, 2>(a.cf, o, nb, __ldcg(bsrc + c)) - nb.c;
    if constexpr (OPK == OP_VARK) d = d / o.d;
    acc[0] += widen(d) * widen(d);
  }
  block_sum<1>(acc, sh);
  const double sc = (OPK == OP_VARK) ? 1.0 : a.dscale2;
  return sqrt(acc[0] * sc / bb);
}

template <typename T, int OPK>
__global__ void __launch_bounds__(1024) k_gs2d(GsArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double sh[32 * MAX_SCAL];
  T* xs = reinterpret_cast<T*>(smraw);
  const int N = (int)a.g.N;
  const T* bsrc = (OPK == OP_VARK) ? a.b : a.bD;
  double acc[1] = {0.0};
  for (int c = threadIdx.x; c < N; c += blockDim.x) {
    const T bv = a.b[c];
    if (OPK != OP_VARK) a.bD[c] = bv * a.invd;
    acc[0] += widen(bv) * widen(bv);
    xs[c] = a.x[c];
  }
  block_sum<1>(acc, sh);   // its barriers also publish bD and xs to the block
  const double bb = acc[0];
  Ctrl* ctrl = a.cm.ctrl;
  if (bb == 0.0) {
    for (int c = threadIdx.x; c < N; c += blockDim.x) a.x[c] = T(0);
    if (threadIdx.x == 0) {
      a.cm.hist[0] = 0.0;
      ctrl->iters = 0;
      ctrl->rel_res = 0.0;
      atomicCAS(&ctrl->status, 0, (int)DS_CONVERGED);
    }
    return;
  }
  int done = 0, status = DS_CONVERGED;
  double rel = -1.0;
  if (a.tol > 0.0) {
    rel = gs2d_residual<T, OPK>(a, xs, bsrc, sh, bb);
    if (threadIdx.x == 0) a.cm.hist[0] = rel;
    status = !(rel > a.tol) ? (isfinite(rel) ? DS_CONVERGED : DS_NONFINITE) : DS_MAXIT;
  }
  if (!(a.tol > 0.0) || status == DS_MAXIT) {
    while (done < a.maxit) {
      const int nb = (a.tol > 0.0) ? min(a.check_every, a.maxit - done) : a.maxit - done;
      if (a.mode == HS_GS_SYMMETRIC) {
        for (int q = 0; q < nb; q++) {
          gs2d_batch<T, OPK>(a, xs, bsrc, 1, false);
          gs2d_batch<T, OPK>(a, xs, bsrc, 1, true);
        }
      } else {
        gs2d_batch<T, OPK>(a, xs, bsrc, nb, a.mode == HS_GS_BACKWARD);
      }
      done += nb;
      if (a.tol > 0.0) {
        rel = gs2d_residual<T, OPK>(a, xs, bsrc, sh, bb);
        if (threadIdx.x == 0) {
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
  for (int c = threadIdx.x; c < N; c += blockDim.x) a.x[c] = xs[c];
  if (threadIdx.x == 0) {
    ctrl->iters = done;
    ctrl->rel_res = rel;
    atomicCAS(&ctrl->status, 0, status);
  }
}

// ---------------------------------------------------------------------------
// Small 2-D grids on one thread-block cluster: the iterate is split by rows
// over the cluster's CTAs (CTA c holds rows [c R, (c + 1) R) in its shared
// memory), the anti-diagonal wavefront and sweep pipelining of k_gs2d run
// unchanged, a node's south / north neighbour in another CTA is read from
// that CTA's shared memory through the cluster's distributed shared memory,
// and the cluster barrier replaces the block barrier after each step.  The
// same update (gs2d_node's gs_old then gs_new) on every node, so the iterates
// are bitwise those of the one-block kernel.
// ---------------------------------------------------------------------------

constexpr int GS2DC_CTAS = 8;   // CTAs per cluster (portable cluster size)

template <typename T, int OPK>
__device__ __forceinline__ void gs2dc_node(const GsArgs<T>& a, T* xs, const T* xlo, const T* xhi, int r0, int r1,
                                           T bv, int i, int j, bool bw) {
  const Geom& g = a.g;
  const int nx = g.nx, ny = g.ny;
  const int cl = (j - r0) * nx + i;   // local index in this CTA's rows
  const T vW = i > 0 ? xs[cl - 1] : T(0);
  const T vE = i + 1 < nx ? xs[cl + 1] : T(0);
  // rows j - 1 and j + 1: this CTA's, or the last row of the CTA below /
  // the first row of the CTA above (distributed shared memory)
  const T vS = j == 0 ? T(0) : (j - 1 >= r0 ? xs[cl - nx] : xlo[i]);
  const T vN = j + 1 >= ny ? T(0) : (j + 1 < r1 ? xs[cl + nx] : xhi[i]);
  const OpRaw<T, OPK> o = op_fetch<T, OPK, 2>(a.cf, g, (long long)j * nx + i, i, j, 0);
  const T yold = gs_old<T, OPK, 2>(a.cf, o, bv, bw ? vW : vE, bw ? vS : vN, T(0), bw);
  xs[cl] = gs_new<T, OPK, 2>(a.cf, o, yold, bw ? vE : vW, bw ? vN : vS, T(0), bw);
}

// Deterministic sum over the cluster: each CTA's block sum, then rank 0 adds
// the CTAs' partials in rank order and every CTA reads the total.
template <typename T>
__device__ double gs2dc_sum(double v, double* sh, double* slot) {
  namespace cgr = cooperative_groups;
  cgr::cluster_group cl = cgr::this_cluster();
  double acc[1] = {v};
  block_sum<1>(acc, sh);
  if (threadIdx.x == 0) slot[0] = acc[0];
  cl.sync();
  if (cl.block_rank() == 0 && threadIdx.x == 0) {
    double t = 0.0;
    for (unsigned r = 0; r < cl.num_blocks(); r++) t += *cl.map_shared_rank(slot, r);
    slot[1] = t;
  }
  cl.sync();
  const double total = *cl.map_shared_rank(slot + 1, 0);
  cl.sync();   // rank 0's slot may be reused only after everyone has read it
  return total;
}

template <typename T, int OPK>
__global__ void __launch_bounds__(1024) k_gs2dc(GsArgs<T> a) {
  namespace cgr = cooperative_groups;
  cgr::cluster_group cl = cgr::this_cluster();
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double sh[32 * MAX_SCAL];
  __shared__ double slot[2];
  T* xs = reinterpret_cast<T*>(smraw);
  const Geom& g = a.g;
  const int nx = g.nx, ny = g.ny;
  const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int R = (ny + C - 1) / C;
  const int r0 = min(ny, rank * R), r1 = min(ny, r0 + R);
  const int nloc = (r1 - r0) * nx;
  // the neighbouring CTAs' rows next to ours (only read when they exist)
  const T* xlo = rank > 0 ? cl.map_shared_rank(xs, rank - 1) + (R - 1) * nx : xs;
  const T* xhi = rank + 1 < C ? cl.map_shared_rank(xs, rank + 1) : xs;
  const T* bsrc = (OPK == OP_VARK) ? a.b : a.bD;
  double acc = 0.0;
  for (int q = threadIdx.x; q < nloc; q += blockDim.x) {
    const long long gi = (long long)r0 * nx + q;
    const T bv = a.b[gi];
    if (OPK != OP_VARK) a.bD[gi] = bv * a.invd;
    acc += widen(bv) * widen(bv);
    xs[q] = a.x[gi];
  }
  __syncthreads();
  const double bb = gs2dc_sum<T>(acc, sh, slot);   // its cluster barriers also publish xs
  Ctrl* ctrl = a.cm.ctrl;
  const bool lead = rank == 0 && threadIdx.x == 0;
  if (bb == 0.0) {
    for (int q = threadIdx.x; q < nloc; q += blockDim.x) a.x[(long long)r0 * nx + q] = T(0);
    if (lead) {
      a.cm.hist[0] = 0.0;
      ctrl->iters = 0;
      ctrl->rel_res = 0.0;
      atomicCAS(&ctrl->status, 0, (int)DS_CONVERGED);
    }
    return;
  }
  // relative residual of the iterate through the Jacobi form (own rows)
  auto residual = [&]() {
    double r = 0.0;
    for (int q = threadIdx.x; q < nloc; q += blockDim.x) {
      const int i = q % nx, j = r0 + q / nx;
      Nbr<T> nb;
      nb.c = xs[q];
      nb.w = i > 0 ? xs[q - 1] : T(0);
      nb.e = i + 1 < nx ? xs[q + 1] : T(0);
      nb.s = j == 0 ? T(0) : (j - 1 >= r0 ? xs[q - nx] : xlo[i]);
      nb.n = j + 1 >= ny ? T(0) : (j + 1 < r1 ? xs[q + nx] : xhi[i]);
      nb.b = nb.t = T(0);
      const long long gi = (long long)j * nx + i;
      const OpRaw<T, OPK> o = op_fetch<T, OPK, 2>(a.cf, g, gi, i, j, 0);
      T d = jacobi_apply<T, OPK, 2>(a.cf, o, nb, __ldcg(bsrc + gi)) - nb.c;
      if constexpr (OPK == OP_VARK) d = d / o.d;
      r += widen(d) * widen(d);
    }
    const double sc = (OPK == OP_VARK) ? 1.0 : a.dscale2;
    return sqrt(gs2dc_sum<T>(r, sh, slot) * sc / bb);
  };
  // nsw sweeps of one direction, pipelined two diagonals apart
  auto batch = [&](int nsw, bool bw) {
    const int Q = blockDim.x / nx;
    const int i = threadIdx.x % nx, q = threadIdx.x / nx;
    const bool active = q < Q;
    const int nsteps = (nx + ny - 2) + 1 + 2 * (nsw - 1);
    const int ii = bw ? nx - 1 - i : i;
    // this CTA's rows in the sweep's frame
    const int f0 = bw ? ny - r1 : r0, f1 = bw ? ny - r0 : r1;
    for (int s = 0; s < nsteps; s++) {
      if (active && f1 > f0) {
        const int t_lo = max(0, (s - i - f1 + 2) >> 1);
        const int t_hi = min(nsw - 1, (s - i - f0) >> 1);
        for (int t = t_lo + (((q - t_lo) % Q) + Q) % Q; t <= t_hi; t += Q) {
          const int r = s - 2 * t - i;
          if (r < f0 || r >= f1) continue;
          const int jj = bw ? ny - 1 - r : r;
          gs2dc_node<T, OPK>(a, xs, xlo, xhi, r0, r1, __ldcg(bsrc + (long long)jj * nx + ii), ii, jj, bw);
        }
      }
      cl.sync();
    }
  };
  int done = 0, status = DS_CONVERGED;
  double rel = -1.0;
  if (a.tol > 0.0) {
    rel = residual();
    if (lead) a.cm.hist[0] = rel;
    status = !(rel > a.tol) ? (isfinite(rel) ? DS_CONVERGED : DS_NONFINITE) : DS_MAXIT;
  }
  if (!(a.tol > 0.0) || status == DS_MAXIT) {
    while (done < a.maxit) {
      const int nb = (a.tol > 0.0) ? min(a.check_every, a.maxit - done) : a.maxit - done;
      if (a.mode == HS_GS_SYMMETRIC) {
        for (int q = 0; q < nb; q++) {
          batch(1, false);
          batch(1, true);
        }
      } else {
        batch(nb, a.mode == HS_GS_BACKWARD);
      }
      done += nb;
      if (a.tol > 0.0) {
        rel = residual();
        if (lead) {
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
  for (int q = threadIdx.x; q < nloc; q += blockDim.x) a.x[(long long)r0 * nx + q] = xs[q];
  if (lead) {
    ctrl->iters = done;
    ctrl->rel_res = rel;
    atomicCAS(&ctrl->status, 0, status);
  }
  cl.sync();   // no CTA leaves while another may still read its rows
}


// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

// Variable coefficients: D, ax, ay, az follow the tile-plane tables, per-tile
// sweep counts and claim counter (sized for the larger tile table), as in the
// tile schedule's workspace.
template <typename T>
static void carve_vark(Carve& c, const hs_op* A, long long N, T** D, T** ax, T** ay, T** az) {
  int nt, P;
  gs_counts(A, &nt, &P);
  c.take<int>((size_t)nt + P + 1);
  c.take<unsigned>((size_t)nt);
  c.take<unsigned long long>(1);
  *D = c.take<T>(N);
  *ax = c.take<T>(N);
  *ay = c.take<T>(N);
  *az = c.take<T>(N);
}

// Largest iterate the single-block 2-D path holds in shared memory.
constexpr size_t GS2D_SMEM_MAX = 200 * 1024;

template <typename T>
static bool gs2d_applies_t(const hs_op* A, const hs_opts& o) {
  if (A->ndim > 2 || A->n[0] > 1024) return false;
  if (o.max_blocks > 1) return false;   // a caller asking for several blocks gets the tile schedule
  const size_t N = (size_t)(A->n[0] * A->n[1]);
  return N * sizeof(T) <= GS2D_SMEM_MAX;
}

template <typename T, int OPK>
static hs_status gs2d_run_t(const SolveArgs& sa, hs_result* res, double* hist) {
  const hs_op* A = sa.A;
  Geom g = geom_of(A);
  Carve c{sa.ws, 0, sa.ws_bytes, true};
  Common cm = carve_common(c, sa.maxit);
  GsArgs<T> a = {};
  a.bD = c.take<T>(g.N);
  T *D = nullptr, *ax = nullptr, *ay = nullptr, *az = nullptr;
  if (OPK == OP_VARK) carve_vark(c, A, g.N, &D, &ax, &ay, &az);
  if (!c.ok) {
    set_error("workspace too small for Gauss-Seidel");
    return HS_ERR_WORKSPACE;
  }
  hs_status s = gs_setup<T, OPK>(sa, cm, D, ax, ay, az, a);
  if (s != HS_OK) return s;
  const size_t smem = (size_t)g.N * sizeof(T);
  auto kern = k_gs2d<T, OPK>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(smem, 1));
  if (e != cudaSuccess) return cuda_fail(e, "shared-memory attribute");
  // Q sweep lanes per column: as many whole columns of threads as fit,
  // rounded up to whole warps (the block reductions use full-warp shuffles;
  // the few extra threads have q = Q and stay idle in the sweeps)
  const int nx = g.nx;
  const int threads = std::min(1024, (((1024 / nx) * nx + 31) / 32) * 32);
  kern<<<1, threads, smem, sa.stream>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "Gauss-Seidel launch");
  return gs_finish<T, OPK>(sa, cm, a, D, ax, ay, az, res, hist);
}

// The cluster form: 2-D grids of at least two rows per CTA whose rows fit the
// CTAs' shared memory, unless the caller caps the grid (max_blocks = 1: one
// block; more: the tile schedule).
template <typename T>
static bool gs2dc_applies_t(const hs_op* A, const hs_opts& o) {
  if (A->ndim != 2 || A->n[0] > 1024 || o.max_blocks != 0) return false;
  const long long nx = A->n[0], ny = A->n[1];
  if (ny < 2 * GS2DC_CTAS) return false;
  const long long R = (ny + GS2DC_CTAS - 1) / GS2DC_CTAS;
  return (size_t)(R * nx) * sizeof(T) <= GS2D_SMEM_MAX;
}

template <typename T, int OPK>
static hs_status gs2dc_run_t(const SolveArgs& sa, hs_result* res, double* hist) {
  const hs_op* A = sa.A;
  Geom g = geom_of(A);
  Carve c{sa.ws, 0, sa.ws_bytes, true};
  Common cm = carve_common(c, sa.maxit);
  GsArgs<T> a = {};
  a.bD = c.take<T>(g.N);
  T *D = nullptr, *ax = nullptr, *ay = nullptr, *az = nullptr;
  if (OPK == OP_VARK) carve_vark(c, A, g.N, &D, &ax, &ay, &az);
  if (!c.ok) {
    set_error("workspace too small for Gauss-Seidel");
    return HS_ERR_WORKSPACE;
  }
  hs_status s = gs_setup<T, OPK>(sa, cm, D, ax, ay, az, a);
  if (s != HS_OK) return s;
  const int nx = g.nx, ny = g.ny;
  const int R = (ny + GS2DC_CTAS - 1) / GS2DC_CTAS;
  const size_t smem = (size_t)R * nx * sizeof(T);
  auto kern = k_gs2dc<T, OPK>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "shared-memory attribute");
  const int threads = std::min(1024, (((1024 / nx) * nx + 31) / 32) * 32);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(GS2DC_CTAS);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = sa.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = GS2DC_CTAS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, kern, a);
  if (e != cudaSuccess) return cuda_fail(e, "Gauss-Seidel cluster launch");
  return gs_finish<T, OPK>(sa, cm, a, D, ax, ay, az, res, hist);
}

bool gs2d_applies(const SolveArgs& sa) {
  return sa.dtype == HS_F64 ? gs2d_applies_t<double>(sa.A, sa.o) : gs2d_applies_t<float>(sa.A, sa.o);
}

bool gs2dc_applies(const SolveArgs& sa) {
  return sa.dtype == HS_F64 ? gs2dc_applies_t<double>(sa.A, sa.o) : gs2dc_applies_t<float>(sa.A, sa.o);
}

#define HS_GS2D(RUN, TT, OK) \
  if (opk == OK) return RUN<TT, OK>(sa, res, hist);

hs_status run_gs2d(const SolveArgs& sa, hs_result* res, double* hist) {
  const int opk = opkind_of(sa.A);
  if (sa.dtype == HS_F64) {
    HS_GS2D(gs2d_run_t, double, OP_SYM)
    HS_GS2D(gs2d_run_t, double, OP_NONSYM)
    HS_GS2D(gs2d_run_t, double, OP_VARK)
  } else {
    HS_GS2D(gs2d_run_t, float, OP_SYM)
    HS_GS2D(gs2d_run_t, float, OP_NONSYM)
    HS_GS2D(gs2d_run_t, float, OP_VARK)
  }
  set_error("unsupported operator");
  return HS_ERR_INVALID;
}

hs_status run_gs2dc(const SolveArgs& sa, hs_result* res, double* hist) {
  const int opk = opkind_of(sa.A);
  if (sa.dtype == HS_F64) {
    HS_GS2D(gs2dc_run_t, double, OP_SYM)
    HS_GS2D(gs2dc_run_t, double, OP_NONSYM)
    HS_GS2D(gs2dc_run_t, double, OP_VARK)
  } else {
    HS_GS2D(gs2dc_run_t, float, OP_SYM)
    HS_GS2D(gs2dc_run_t, float, OP_NONSYM)
    HS_GS2D(gs2dc_run_t, float, OP_VARK)
  }
  set_error("unsupported operator");
  return HS_ERR_INVALID;
}

#undef HS_GS2D

}  // namespace hs
