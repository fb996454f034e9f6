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
//
// Single sweeps and the symmetric method on grids whose x-y plane fits in
// shared memory take a second schedule, k_gs27p: whole planes per block,
// pipelined along z four in-plane steps apart (below).  Both apply the same
// update (gs27_update), so their iterates agree bitwise.
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
  int R;            // rem steps per plane (plane-lagged schedule)
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

// The 27-point update split by z plane, in the order both schedules use (so
// their iterates agree bitwise): the 3 x 3 block q of one plane sums its ring
// of 8 around the column, then the column node q[4]; x_i = (b_i + (dn + up)
// + ring) / 27 with dn / up the 9-sums of the planes below / above and ring
// the 8 in-plane neighbours, formed as fma(1/27, ., b_i / 27).
template <typename T>
__device__ __forceinline__ T gs27_ring(const T* q) {
  return ((q[0] + q[1]) + (q[2] + q[3])) + ((q[5] + q[6]) + (q[7] + q[8]));
}

template <typename T>
__device__ __forceinline__ T gs27_finish(T dn, T up, T ring, T bD, T g27) {
  return fma(g27, (dn + up) + ring, bD);
}

// From the 3 x 3 x 3 box v (center unused) and bD = b_i / 27.
template <typename T>
__device__ __forceinline__ T gs27_update(const T (&v)[27], T bD, T g27) {
  return gs27_finish(gs27_ring(v) + v[4], gs27_ring(v + 18) + v[22], gs27_ring(v + 9), bD, g27);
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
  a.x[idx] = gs27_update(v, __ldcg(a.bD + idx), a.g27);
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

// The solve both 27-point kernels run: b / 27 and ||b||^2, the initial
// residual, batches of sweeps (batch(nsw, backward) sweeps nsw times in one
// direction and returns false when the solve has to stop), the residual after
// each batch, the final status.  The caller zeroes its progress words first;
// the first reduction orders that before any wait.
template <typename T, class Batch>
__device__ __forceinline__ void gs27_solve(const Gs27Args<T>& a, double* sh, Batch&& batch) {
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
          if (!batch(1, false)) return;
          if (!batch(1, true)) return;
        }
      } else {
        if (!batch(nb, a.mode == HS_GS_BACKWARD)) return;
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
__global__ void __launch_bounds__(GS27_THREADS) k_gs27(Gs27Args<T> a) {
  __shared__ double sh[32 * MAX_SCAL];
  if (threadIdx.x == 0) a.prog[blockIdx.x] = 0;
  unsigned long long base = 0;
  gs27_solve(a, sh, [&](int nsw, bool bw) { return gs27_batch(a, base, nsw, bw); });
}

// ---------------------------------------------------------------------------
// Plane-lagged schedule (grids whose x-y plane fits in shared memory).  A
// block owns whole z planes (plane k to block k mod G) and sweeps one plane
// at a time, staged in shared memory, in the in-plane order rem = i + 2j:
// the in-plane lower neighbours of a node lie on rem - 1 .. rem - 3, so the
// nodes of one rem are independent (one block barrier per rem step).  Node
// (i, j) of plane k at rem r reads, from the plane below, nodes at rem r - 3
// .. r + 3 (h - 7 .. h - 1 in the hyperplane numbering), which must hold the
// current sweep's values, and from the plane above nodes of the same range,
// which must still hold the previous sweep's.  So sweep t starts on plane k
// once sweep t - 1 has finished plane k + 1, and runs rem r once sweep t has
// finished rem r + 3 on plane k - 1; the planes form a pipeline four rem
// steps apart, with no grid-wide step.  Each plane publishes t R + (rems
// done) (R rems per plane; monotonic over sweeps) every GS27P_PUB steps and
// at its end.  The last warp of the block does the publishing and the
// polling of the new-side plane, off the path of the rem steps; the compute
// warps load each step's operands a step ahead (so a rem step waits for
// rem r + 4 of the plane below, one more than the data needs) and work two
// lanes per node.  On this GPU a rem step is bound by its SM's FP64 pipes
// (about 27 operations per node, 0.5 lane per clock on each of the four SM
// sub-partitions): the pair of lanes puts a 64-node step on four warps
// instead of two (128 x 128 x 6144, one sweep: 72 against 89 ms with one
// lane per node, 106 ms for the hyperplane schedule).  A backward sweep
// mirrors i, j and k.  Every block takes its
// items (t, k) in the order of sweeps and, within a sweep, of its planes in
// the sweep's direction; an item waits only on earlier items, so the
// earliest unfinished one can always proceed: no deadlock, whatever the
// interleaving.  A single sweep takes about n_z four-rem lags instead of
// n_x + 2 n_y + 4 n_z grid-wide hyperplane steps.
// ---------------------------------------------------------------------------

#ifndef HS_GS27P_PUB
#define HS_GS27P_PUB 1
#endif
constexpr int GS27P_PUB = HS_GS27P_PUB;       // rem steps between publications
constexpr size_t GS27P_SMEM_MAX = 200 * 1024;  // largest staged plane
// progress words 128 bytes apart: each in a cache line of its own
constexpr int GS27P_PSTRIDE = 16;

// One thread: wait until *p >= target, bounded by the solve's timeout (status
// DS_TIMEOUT); ends early when another block has flagged an error.  The last
// value read goes to *seen.
__device__ __forceinline__ bool wait_count(const unsigned long long* p, unsigned long long target, Ctrl* ctrl,
                                           unsigned long long* seen) {
  unsigned spins = 0;
  unsigned long long t0 = 0, v;
  while ((v = ld_acquire_u64(p)) < target) {
    if ((++spins & 1023) == 0) {
      if (t0 == 0) t0 = global_ns();
      if (ld_acquire_int(&ctrl->status) < 0) return false;
      if (global_ns() - t0 > ctrl->timeout_ns) {
        atomicCAS(&ctrl->status, 0, (int)DS_TIMEOUT);
        return false;
      }
    }
  }
  *seen = v;
  return true;
}

// The 3 x 3 block of plane kk around column (i, j), zeros outside the grid
// (its 9-sum is gs27_ring(q) + q[4]).
template <typename T>
__device__ __forceinline__ void gs27p_load9(const Gs27Args<T>& a, int i, int j, int kk, T (&q)[9]) {
  const Geom& g = a.g;
  const int nx = g.nx;
  const bool okz = kk >= 0 && kk < g.nz;
  const long long idx = (long long)kk * g.plane + (long long)j * nx + i;
  const bool okx[3] = {i > 0, true, i + 1 < nx};
  const bool oky[3] = {j > 0, true, j + 1 < g.ny};
#pragma unroll
  for (int dy = 0; dy < 3; dy++)
#pragma unroll
    for (int dx = 0; dx < 3; dx++) {
      const long long at = idx + (long long)(dy - 1) * nx + (dx - 1);
      q[dy * 3 + dx] = (okz && oky[dy] && okx[dx] && HS_IN_BOUNDS(at, g.N)) ? __ldcg(a.x + at) : T(0);
    }
}

// The 8 in-plane neighbours of (i, j) in the staged plane, as gs27_ring.
template <typename T>
__device__ __forceinline__ T gs27p_inplane(const T* xs, int nx, int ny, int i, int j) {
  const int c = j * nx + i;
  const bool okx[3] = {i > 0, true, i + 1 < nx};
  const bool oky[3] = {j > 0, true, j + 1 < ny};
  T q[9];
#pragma unroll
  for (int dy = 0; dy < 3; dy++)
#pragma unroll
    for (int dx = 0; dx < 3; dx++)
      q[dy * 3 + dx] = (oky[dy] && okx[dx] && !(dy == 1 && dx == 1)) ? xs[c + (dy - 1) * nx + (dx - 1)] : T(0);
  return gs27_ring(q);
}

// Named barrier 1: the compute warps of a block (all but the last warp).
__device__ __forceinline__ void bar_compute(int nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// Compute thread 0: wait until the new-side count the sync warp has seen
// reaches `need`.  Ends when the sync warp gives up (s_fail) and, as a
// backstop, after twice the solve's timeout.
__device__ __forceinline__ bool gs27p_wait_seen(const volatile unsigned long long* s_seen, volatile int* s_fail,
                                                unsigned long long need, Ctrl* ctrl) {
  unsigned spins = 0;
  unsigned long long t0 = 0;
  while (*s_seen < need) {
    if (*s_fail) return false;
    if ((++spins & 1023) == 0) {
      if (t0 == 0) {
        t0 = global_ns();
      } else if (global_ns() - t0 > 2 * ctrl->timeout_ns) {
        atomicCAS(&ctrl->status, 0, (int)DS_TIMEOUT);
        *s_fail = 1;
        return false;
      }
    }
  }
  __threadfence_block();
  return true;
}

// The sync warp's lane 0 during one plane: publishes the rem steps the
// compute warps report done (s_done, every GS27P_PUB steps and at the end:
// release store of t R + steps) and keeps reading the new-side plane's count
// into s_seen, so that neither a publication nor a poll sits between two rem
// steps.  Gives up (s_fail, status DS_TIMEOUT) when nothing has moved for
// the solve's timeout, or when another block has flagged an error.
template <typename T>
__device__ void gs27p_sync(const Gs27Args<T>& a, int k, int kp, bool has_p, unsigned long long tR, int R,
                           volatile unsigned long long* s_seen, const volatile int* s_done, volatile int* s_fail) {
  Ctrl* ctrl = a.cm.ctrl;
  const unsigned long long full = tR + (unsigned long long)R;
  unsigned long long seen = has_p ? 0ull : full;
  unsigned long long t0 = global_ns();
  unsigned spins = 0;
  int pub = 0;
  while (true) {
    const int d = *s_done;
    bool moved = false;
    if (d != pub && (d - pub >= GS27P_PUB || d == R)) {
      __threadfence_block();
      st_release_u64(a.prog + (long long)k * GS27P_PSTRIDE, tR + (unsigned long long)d);
      pub = d;
      moved = true;
    }
    if (pub == R || *s_fail) return;
    if (seen < full) {
      const unsigned long long v = ld_acquire_u64(a.prog + (long long)kp * GS27P_PSTRIDE);
      if (v > seen) {
        seen = v;
        __threadfence_block();
        *s_seen = v;
        moved = true;
      }
    }
    if (moved) {
      t0 = global_ns();
      spins = 0;
    } else if ((++spins & 255) == 0) {
      if (ld_acquire_int(&ctrl->status) < 0) {
        *s_fail = 1;
        return;
      }
      if (global_ns() - t0 > ctrl->timeout_ns) {
        atomicCAS(&ctrl->status, 0, (int)DS_TIMEOUT);
        *s_fail = 1;
        return;
      }
    }
  }
}

// Two compute lanes per node (lanes 2m, 2m + 1 of a warp: node m of the rem
// step), so that a step's FP64 work spreads over twice the warps: lane 0 of
// the pair sums the new-side plane's 3 x 3 block and the in-plane neighbours
// of the row below (and the west one), lane 1 the old-side block and the
// other four, with b / 27; lane 0 combines them.  The operands of the next
// step are loaded a step ahead.
template <typename T>
struct Gs27pSlot {
  bool act;
  int i, j, c;    // node and its position in the plane
  long long idx;  // position in the grid
  T v[9], bD;     // the pair lane's plane block; b / 27 (lane 1)
};

// Issue rem r's loads for pair lane (m, side) into `sl` (the new-side plane
// must have published rems up to r + 3 of this sweep).
template <typename T>
__device__ __forceinline__ void gs27p_fetch(const Gs27Args<T>& a, int r, int m, int side, bool bw, int k, int kn,
                                           int kp, Gs27pSlot<T>& sl) {
  const Geom& g = a.g;
  const int nx = g.nx, ny = g.ny;
  const int jlo = r - nx + 1 > 0 ? (r - nx + 2) / 2 : 0;
  const int jf = jlo + m;
  sl.act = r < a.R && jf <= min(ny - 1, r / 2);
  const int i = bw ? nx - 1 - (r - 2 * jf) : r - 2 * jf;
  const int j = bw ? ny - 1 - jf : jf;
  sl.i = i;
  sl.j = j;
  sl.c = j * nx + i;
  sl.idx = (long long)k * g.plane + sl.c;
  if (sl.act && HS_IN_BOUNDS(sl.idx, g.N)) {
    gs27p_load9(a, i, j, side ? kn : kp, sl.v);
    sl.bD = side ? __ldcg(a.bD + sl.idx) : T(0);
  } else {
    sl.act = false;
    sl.bD = T(0);
  }
}

// Update the pair's node.  Every compute lane calls it (warp shuffles).
template <typename T>
__device__ __forceinline__ void gs27p_apply(const Gs27Args<T>& a, T* xs, const Gs27pSlot<T>& sl, int side) {
  const int nx = a.g.nx, ny = a.g.ny;
  T s9 = T(0), h = T(0);
  if (sl.act) {
    const int i = sl.i, j = sl.j;
    // in-plane block positions of this lane: 0..3 (side 0) or 5..8 (side 1)
    T q[4];
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const int p = side ? e + 5 : e;
      const int dy = p / 3 - 1, dx = p % 3 - 1;
      const bool ok = (j + dy >= 0) && (j + dy < ny) && (i + dx >= 0) && (i + dx < nx);
      q[e] = ok ? xs[sl.c + dy * nx + dx] : T(0);
    }
    s9 = gs27_ring(sl.v) + sl.v[4];
    h = (q[0] + q[1]) + (q[2] + q[3]);
  }
  const T o9 = __shfl_xor_sync(0xffffffffu, s9, 1);
  const T oh = __shfl_xor_sync(0xffffffffu, h, 1);
  const T obD = __shfl_xor_sync(0xffffffffu, sl.bD, 1);
  if (sl.act && side == 0) {
    // (dn + up) is symmetric; the ring is gs27_ring's ((0+1)+(2+3)) + ((5+6)+(7+8))
    const T xn = fma(a.g27, (s9 + o9) + (h + oh), obD);
    xs[sl.c] = xn;
    a.x[sl.idx] = xn;
  }
}

// Sweep t (counted from the start of the solve) of plane k.  The last warp
// of the block waits and publishes (gs27p_sync); the others stage the plane
// and sweep it, one named barrier per rem step.  Compute thread 0 checks,
// before each barrier, that the new-side plane is far enough for the loads
// the next step issues and writes the outcome to s_stop[parity of that
// step], which every compute thread reads after the barrier: all of them
// leave the loop at the same step.
template <typename T>
__device__ bool gs27p_plane(const Gs27Args<T>& a, T* xs, int k, unsigned long long t, bool bw) {
  __shared__ int s_ok;
  __shared__ int s_stop[2];
  __shared__ volatile int s_done;
  __shared__ volatile int s_fail;
  __shared__ volatile unsigned long long s_seen;
  const Geom& g = a.g;
  const int nx = g.nx, ny = g.ny, npl = nx * ny, R = a.R;
  const unsigned long long tR = t * (unsigned long long)R;
  const int kp = bw ? k + 1 : k - 1;   // new side: swept before plane k
  const int kn = bw ? k - 1 : k + 1;   // old side: must hold sweep t - 1
  const bool has_p = kp >= 0 && kp < g.nz;
  const bool has_n = kn >= 0 && kn < g.nz;
  const int nct = (int)blockDim.x - 32;
  const int q = threadIdx.x;
  if (q == nct) {
    unsigned long long v = 0;
    s_ok = (!has_n || wait_count(a.prog + (long long)kn * GS27P_PSTRIDE, tR, a.cm.ctrl, &v)) ? 1 : 0;
    s_seen = has_p ? 0ull : ~0ull;
    s_done = 0;
    s_fail = 0;
    s_stop[0] = 0;
    s_stop[1] = 0;
  }
  // this block swept plane k last (or it holds the initial iterate)
  const T* xk = a.x + (long long)k * g.plane;
  if (q < nct)
    for (int c = q; c < npl; c += nct) xs[c] = __ldcg(xk + c);
  __syncthreads();
  if (!s_ok) return false;
  if (q >= nct) {
    if (q == nct) gs27p_sync(a, k, kp, has_p, tR, R, &s_seen, &s_done, &s_fail);
  } else {
    // operands are loaded one step ahead (two register slots, rotated by
    // unrolling): before the barrier that ends step r, thread 0 waits until
    // the new-side plane has published rem r + 5, the last one the loads of
    // step r + 2 read
    auto need_of = [&](int r) { return has_p ? tR + (unsigned long long)min(r + 4, R) : 0ull; };
    Gs27pSlot<T> A, B;
    if (q == 0 && !gs27p_wait_seen(&s_seen, &s_fail, need_of(1), a.cm.ctrl)) s_stop[0] = 1;
    bar_compute(nct);
    int r = 0;
    if (!s_stop[0]) gs27p_fetch(a, 0, q >> 1, q & 1, bw, k, kn, kp, A);
    // one rem step: load step r + 1 into `nxt`, update from `cur`; false
    // when the solve has to stop or the plane is done (the same answer in
    // every compute thread)
    auto step = [&](Gs27pSlot<T>& cur, Gs27pSlot<T>& nxt) -> bool {
      if (s_stop[r & 1]) return false;
      if (r + 1 < R) gs27p_fetch(a, r + 1, q >> 1, q & 1, bw, k, kn, kp, nxt);
      gs27p_apply(a, xs, cur, q & 1);
      if (q == 0 && r + 2 < R && !gs27p_wait_seen(&s_seen, &s_fail, need_of(r + 2), a.cm.ctrl))
        s_stop[(r + 1) & 1] = 1;
      bar_compute(nct);
      if (q == 0) {
        __threadfence_block();
        s_done = r + 1;
      }
      r++;
      return r < R;
    };
    while (step(A, B) && step(B, A)) {
    }
  }
  __syncthreads();
  return !s_fail;
}

// nsw sweeps of one direction; tsw counts the sweeps done before (the same
// in every block).
template <typename T>
__device__ bool gs27p_batch(const Gs27Args<T>& a, T* xs, unsigned long long& tsw, int nsw, bool bw) {
  const int nz = a.g.nz, G = gridDim.x, b = blockIdx.x;
  if (b < nz) {
    const int ktop = b + G * ((nz - 1 - b) / G);   // highest plane of this block
    for (int s = 0; s < nsw; s++) {
      for (int k = bw ? ktop : b; bw ? k >= b : k <= ktop; k += bw ? -G : G)
        if (!gs27p_plane(a, xs, k, tsw + (unsigned long long)s, bw)) return false;
    }
  }
  tsw += (unsigned long long)nsw;
  return true;
}

template <typename T>
__global__ void __launch_bounds__(GS27_THREADS, 1) k_gs27p(Gs27Args<T> a) {
  __shared__ double sh[32 * MAX_SCAL];
  extern __shared__ __align__(16) unsigned char gs27p_smem[];
  T* xs = reinterpret_cast<T*>(gs27p_smem);
  for (int k = blockIdx.x + gridDim.x * (int)threadIdx.x; k < a.g.nz; k += gridDim.x * blockDim.x) a.prog[(long long)k * GS27P_PSTRIDE] = 0;
  unsigned long long tsw = 0;
  gs27_solve(a, sh, [&](int nsw, bool bw) { return gs27p_batch(a, xs, tsw, nsw, bw); });
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

// A plane fits shared memory and each rem has at most one node per pair of
// compute threads (all warps but the last).
template <typename T>
static bool gs27p_fits(const hs_op* A) {
  return (size_t)(A->n[0] * A->n[1]) * sizeof(T) <= GS27P_SMEM_MAX &&
         std::min<long long>(A->n[1], (A->n[0] + 1) / 2) <= (GS27_THREADS - 32) / 2;
}

template <typename T>
static hs_status gs27_t(const SolveArgs& sa, hs_result* res, double* hist) {
  const hs_op* A = sa.A;
  const Geom g = geom_of(A);
  // schedule: the plane-lagged one for single sweeps and the symmetric
  // method (a sweep takes about n_z lags of four rem steps), the hyperplane
  // one for batches of four or more sweeps of one direction, which it
  // pipelines eight hyperplanes apart (the plane-lagged schedule starts a
  // sweep on a plane only after the previous sweep has left the plane above,
  // and each block takes its planes sweep by sweep)
  const int per_batch = sa.tol > 0.0 ? sa.o.check_every : sa.maxit;
  const bool deep = sa.o.gs_mode == HS_GS_SYMMETRIC || per_batch < 4;
  if (sa.o.gs_schedule == 3 || (sa.o.gs_schedule == 2 && !gs27p_fits<T>(A))) {
    set_error(sa.o.gs_schedule == 3 ? "the cluster schedule is for 2-D grids; the 27-point operator is 3-D"
                                    : "the plane-lagged 27-point schedule needs an x-y plane of at most 200 KB with "
                                      "min(n_y, ceil(n_x / 2)) <= 112");
    return HS_ERR_INVALID;
  }
  const bool planes = gs27p_fits<T>(A) && (sa.o.gs_schedule == 2 || (sa.o.gs_schedule == 0 && deep));
  Carve c{sa.ws, 0, sa.ws_bytes, true};
  Common cm = carve_common(c, sa.maxit);
  Gs27Args<T> a = {};
  a.bD = c.take<T>(g.N);
  a.prog = c.take<unsigned long long>(std::max<size_t>(GS27_MAX_BLOCKS, (size_t)g.nz * GS27P_PSTRIDE));
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
  a.R = (g.nx - 1) + 2 * (g.ny - 1) + 1;
  a.M = g.nx / 2 + 1;
  a.maxit = sa.maxit;
  a.mode = sa.o.gs_mode;
  a.check_every = sa.o.check_every;
  a.tol = sa.tol;
  const void* kern = planes ? (const void*)k_gs27p<T> : (const void*)k_gs27<T>;
  const size_t smem = planes ? (size_t)g.plane * sizeof(T) : 0;
  cudaError_t e = cudaSuccess;
  if (planes) {
    e = cudaFuncSetAttribute(k_gs27p<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "shared-memory attribute");
  }
  // one block per SM: a hyperplane holds a few thousand nodes (about 65 per
  // plane), and the plane-lagged pipeline keeps a few dozen planes busy, each
  // bound by its SM's FP64 pipes, so more blocks would only idle or share them
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, GS27_THREADS, smem);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
  if (per_sm < 1) {
    set_error("Gauss-Seidel kernel cannot be resident");
    return HS_ERR_CUDA;
  }
  int grid = std::min(sm_count(), GS27_MAX_BLOCKS);
  if (planes) grid = std::min(grid, g.nz);
  if (sa.o.max_blocks > 0) grid = std::min(grid, sa.o.max_blocks);
  void* args[] = {&a};
  s = launch_coop(kern, grid, GS27_THREADS, args, smem, sa.stream);
  if (s != HS_OK) return s;
  s = hs_dbg_take(sa.stream);
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

// The plane-lagged waits on a plane count that nothing publishes
// (diagnostic): lane 0 of warp 2 waits for an old-side plane (wait_count),
// lane 0 of warp 1 polls a new-side plane (gs27p_sync) and compute thread 0
// waits for the count the poller has seen (gs27p_wait_seen).
__global__ void k_diag_gs27p(Ctrl* ctrl, unsigned long long* words) {
  __shared__ volatile unsigned long long s_seen;
  __shared__ volatile int s_done, s_fail;
  if (threadIdx.x == 0) {
    s_seen = 0;
    s_done = 0;
    s_fail = 0;
  }
  __syncthreads();
  Gs27Args<double> a = {};
  a.prog = words;
  a.cm.ctrl = ctrl;
  if (threadIdx.x == 0) gs27p_wait_seen(&s_seen, &s_fail, 1ull, ctrl);
  if (threadIdx.x == 32) gs27p_sync(a, 1, 0, true, 0ull, 1, &s_seen, &s_done, &s_fail);
  if (threadIdx.x == 64) {
    unsigned long long v = 0;
    wait_count(words + GS27P_PSTRIDE, 1ull, ctrl, &v);
  }
}

hs_status diag_gs27p_wait(Ctrl* ctrl, unsigned long long* words, cudaStream_t st) {
  k_diag_gs27p<<<1, 96, 0, st>>>(ctrl, words);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HS_OK : cuda_fail(e, "diagnostic launch");
}

// Progress words: one per block (hyperplane schedule) or per z plane
// (plane-lagged schedule).
size_t gs27_progress_bytes(const hs_op* A) {
  const size_t words = std::max<size_t>(GS27_MAX_BLOCKS, (size_t)A->n[2] * GS27P_PSTRIDE);
  return (words * sizeof(unsigned long long) + 255) & ~(size_t)255;
}

hs_status run_gauss_seidel27(const SolveArgs& sa, hs_result* res, double* hist) {
  return sa.dtype == HS_F64 ? gs27_t<double>(sa, res, hist) : gs27_t<float>(sa, res, hist);
}

}  // namespace hs
