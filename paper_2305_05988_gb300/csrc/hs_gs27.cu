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
// is one step and nodes are updated in place in global memory.
//
// Consecutive sweeps of one direction are pipelined: sweep t runs hyperplane
// tau - 8t at step tau.  A node's neighbours lie within 7 hyperplanes, so the
// upper neighbours sweep t+1 reads hold sweep t's values and no two active
// hyperplanes of a step touch each other's nodes.
//
// The steps need no grid-wide barrier.  The z planes are dealt to the blocks
// round robin (plane k to block k mod G), and a node of plane k reads planes
// k-1, k and k+1 only, so a block waits before each step until its two ring
// neighbours (the owners of planes k-1 and k+1) have completed the previous
// step, and then publishes its own step count.  Waiting on both sides keeps
// a block from overwriting values a neighbour still has to read (with
// pipelined sweeps the lower plane's next sweep would otherwise catch up);
// a block with no node on the step's hyperplanes publishes without waiting.
// Batches and directions follow one another under the same rule, so a
// backward sweep starts on a plane as soon as its neighbours have finished
// the forward one.
//
// Hyperplane h holds, for each k with a non-empty range, the lines j with
// 0 <= h - 4k - 2j < nx; a block's threads take (sweep, plane, slot) triples
// with M = nx/2 + 1 slots per plane (the longest j range).
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
  unsigned long long* prog;    // per block: steps completed (only grows)
  int H;            // hyperplanes per sweep
  int M;            // slots per k
  int maxit;
  int mode;         // HS_GS_FORWARD / BACKWARD / SYMMETRIC
  int check_every;
  double tol;
};

constexpr int GS27_LAG = 8;
constexpr int GS27_THREADS = 256;
// progress words reserved in the workspace (the grid is at most one block per SM)
constexpr int GS27_MAX_BLOCKS = 1024;

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Thread 0 of a block: wait until both ring neighbours have completed
// `target` steps.  Bounded by the solve's timeout (status DS_TIMEOUT); ends
// early when another block has flagged an error.
__device__ __forceinline__ bool wait_neighbours(const unsigned long long* lo, const unsigned long long* hi,
                                unsigned long long target, Ctrl* ctrl) {
  unsigned spins = 0;
  unsigned long long t0 = 0;
  while (ld_acquire_u64(lo) < target || ld_acquire_u64(hi) < target) {
    if ((++spins & 1023) == 0) {
      if (t0 == 0) t0 = global_ns();
      if (ld_acquire_int(&ctrl->status) < 0) return false;
      if (global_ns() - t0 > ctrl->timeout_ns) {
        atomicCAS(&ctrl->status, 0, (int)DS_TIMEOUT);
        return false;
      }
    }
  }
  return true;
}

// k range of hyperplane h (empty when klo > khi).
__device__ __forceinline__ void gs27_krange(const Geom& g, int h, int& klo, int& khi) {
  khi = min(g.nz - 1, h / 4);
  const int r = h - (g.nx - 1) - 2 * (g.ny - 1);   // 4k >= r
  klo = r <= 0 ? 0 : (r + 3) / 4;
}

// x_i <- (b_i + sum of the 26 neighbours) / 27, in place.  All 26 loads are
// issued before the first addition (nodes outside the grid read as zero).
template <typename T>
__device__ __forceinline__ void gs27_node(const Gs27Args<T>& a, int i, int j, int k) {
  const Geom& g = a.g;
  const long long idx = (long long)k * g.plane + (long long)j * g.nx + i;
  const bool okx[3] = {i > 0, true, i + 1 < g.nx};
  const bool oky[3] = {j > 0, true, j + 1 < g.ny};
  const bool okz[3] = {k > 0, true, k + 1 < g.nz};
  T v[27];
#pragma unroll
  for (int dz = 0; dz < 3; dz++)
#pragma unroll
    for (int dy = 0; dy < 3; dy++)
#pragma unroll
      for (int dx = 0; dx < 3; dx++) {
        const long long off = (long long)(dz - 1) * g.plane + (long long)(dy - 1) * g.nx + (dx - 1);
        const bool center = dz == 1 && dy == 1 && dx == 1;   // not needed
        v[dz * 9 + dy * 3 + dx] = (!center && okz[dz] && oky[dy] && okx[dx]) ? __ldcg(a.x + idx + off) : T(0);
      }
  const T bD = __ldcg(a.bD + idx);
  // ring of each plane (the 8 nodes around the column), then the columns
  T ring[3];
#pragma unroll
  for (int dz = 0; dz < 3; dz++) {
    const T* q = v + dz * 9;
    ring[dz] = ((q[0] + q[1]) + (q[2] + q[3])) + ((q[5] + q[6]) + (q[7] + q[8]));
  }
  const T nbr = ((ring[0] + ring[2]) + ring[1]) + (v[4] + v[22]);
  a.x[idx] = fma(a.g27, nbr, bD);
}

// First plane at or above klo owned by block b of G (plane k belongs to block
// k mod G) and the number of owned planes in [klo, khi].
__device__ __forceinline__ int gs27_owned(int klo, int khi, int b, int G, int& k0) {
  k0 = klo + ((b - klo % G) % G + G) % G;
  return k0 <= khi ? (khi - k0) / G + 1 : 0;
}

// nsw pipelined sweeps of one direction.  `base` counts the steps completed
// before this batch (the same in every block) and advances by the batch's
// step count.
template <typename T>
__device__ __forceinline__ bool gs27_batch(const Gs27Args<T>& a, unsigned long long& base, int nsw, bool backward) {
  __shared__ int s_ok;
  const Geom& g = a.g;
  const int H = a.H, M = a.M;
  const int G = gridDim.x, b = blockIdx.x;
  const unsigned long long* plo = a.prog + (b + G - 1) % G;
  const unsigned long long* phi = a.prog + (b + 1) % G;
  const int nsteps = H + GS27_LAG * (nsw - 1);
  for (int tau = 0; tau < nsteps; tau++) {
    const int t_hi = min(nsw - 1, tau / GS27_LAG);
    // owned work of this step: sweeps t_hi .. t_lo are active
    int total = 0;
    for (int t = t_hi; t >= 0; t--) {
      const int sidx = tau - GS27_LAG * t;
      if (sidx >= H) break;
      const int h = backward ? H - 1 - sidx : sidx;
      int klo, khi, k0;
      gs27_krange(g, h, klo, khi);
      if (klo <= khi) total += gs27_owned(klo, khi, b, G, k0);
    }
    if (total > 0) {
      if (threadIdx.x == 0) s_ok = wait_neighbours(plo, phi, base + tau, a.cm.ctrl);
      __syncthreads();
      if (!s_ok) return false;
      int off = 0;   // first slot index of the current (sweep, plane) group
      for (int t = t_hi; t >= 0; t--) {
        const int sidx = tau - GS27_LAG * t;
        if (sidx >= H) break;
        const int h = backward ? H - 1 - sidx : sidx;
        int klo, khi, k0;
        gs27_krange(g, h, klo, khi);
        if (klo > khi) continue;
        const int cnt = gs27_owned(klo, khi, b, G, k0);
        const int nslot = cnt * M;
        // this thread's slots are those congruent to threadIdx.x mod blockDim.x
        int e = off + ((int)threadIdx.x - off % (int)blockDim.x + (int)blockDim.x) % (int)blockDim.x;
        for (; e < off + nslot; e += blockDim.x) {
          const int loc = e - off;
          const int k = k0 + (loc / M) * G;
          const int rem = h - 4 * k;                       // = i + 2j
          const int jlo = rem - (g.nx - 1) <= 0 ? 0 : (rem - (g.nx - 1) + 1) / 2;
          const int j = jlo + loc % M;
          if (j >= g.ny || 2 * j > rem) continue;
          gs27_node(a, rem - 2 * j, j, k);
        }
        off += nslot;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      __threadfence();
      st_release_u64(a.prog + b, base + tau + 1);
    }
  }
  base += nsteps;
  return true;
}

// Relative residual through the Jacobi form, reduced over the grid.
template <typename T>
__device__ bool gs27_residual(const Gs27Args<T>& a, double* sh, double bb, double* rel) {
  const Geom& g = a.g;
  // blocks finish a batch at different times: all sweeps must be complete
  if (!grid_sync(a.cm.ctrl, a.cm.partials, sh)) return false;
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
__global__ void __launch_bounds__(GS27_THREADS) k_gs27(Gs27Args<T> a) {
  __shared__ double sh[32 * MAX_SCAL];
  const long long N = a.g.N;
  unsigned long long base = 0;
  if (threadIdx.x == 0) a.prog[blockIdx.x] = 0;   // ordered by the reduction below
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
          if (!gs27_batch(a, base, 1, false)) return;
          if (!gs27_batch(a, base, 1, true)) return;
        }
      } else {
        if (!gs27_batch(a, base, nb, a.mode == HS_GS_BACKWARD)) return;
      }
      done += nb;
      if (a.tol > 0.0) {
        if (!gs27_residual(a, sh, bb[0], &rel)) return;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
          for (int q = done - nb + 1; q < done; q++) a.cm.hist[q] = __longlong_as_double(0x7ff8000000000000LL);   // not evaluated (quiet NaN)
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
  a.prog = c.take<unsigned long long>(GS27_MAX_BLOCKS);
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
  // one block per SM: a hyperplane holds a few thousand nodes (about 65 per
  // plane), so more blocks would only idle
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gs27<T>, GS27_THREADS, 0);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
  if (per_sm < 1) {
    set_error("Gauss-Seidel kernel cannot be resident");
    return HS_ERR_CUDA;
  }
  int grid = std::min(sm_count(), GS27_MAX_BLOCKS);
  if (sa.o.max_blocks > 0) grid = std::min(grid, sa.o.max_blocks);
  void* args[] = {&a};
  s = launch_coop((const void*)k_gs27<T>, grid, GS27_THREADS, args, 0, sa.stream);
  if (s != HS_OK) return s;
  return finish_solve_pub(sa, cm, nullptr, nullptr, nullptr, nullptr, a.bD, res, hist, sa.tol > 0.0);
}

// Thread 0 waits for ring neighbours that never publish (diagnostic).
__global__ void k_diag_gs27(Ctrl* ctrl, const unsigned long long* words) {
  if (threadIdx.x == 0) wait_neighbours(words, words + 1, 1ull, ctrl);
}

hs_status diag_gs27_wait(Ctrl* ctrl, const unsigned long long* words, cudaStream_t st) {
  k_diag_gs27<<<1, 32, 0, st>>>(ctrl, words);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HS_OK : cuda_fail(e, "diagnostic launch");
}

size_t gs27_progress_bytes() { return (GS27_MAX_BLOCKS * sizeof(unsigned long long) + 255) & ~(size_t)255; }

hs_status run_gauss_seidel27(const SolveArgs& sa, hs_result* res, double* hist) {
  return sa.dtype == HS_F64 ? gs27_t<double>(sa, res, hist) : gs27_t<float>(sa, res, hist);
}

}  // namespace hs
