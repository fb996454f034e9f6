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
//   * tiles of TX x TY x TZ nodes, tile hyperplane S = I + J + K: a tile
//     needs the current sweep's values of its three lower face neighbours
//     and the previous sweep's of its three upper ones.  The tiles are
//     scheduled as a dataflow graph, not in grid-wide steps: blocks take
//     (sweep, tile) items from a counter in the order of the step schedule
//     (sweep t's tile plane S at step 2t + S, so consecutive sweeps of the
//     same direction overlap) and wait on per-tile sweep counts of the
//     face neighbours before sweeping a tile;
//   * inside a tile (staged in shared memory with a one-node halo), one
//     thread per x-line; the line (j, k) processes node i at local step
//     i + j + k.  Lines are dealt to threads in order of j + k so that the
//     32 lines of a warp start within a few steps of each other and the
//     scarce FP64 pipe is not spent on idle lanes.
//
// A backward sweep mirrors every direction.  The symmetric method (forward
// then backward per iteration) alternates directions inside one batch; a
// sweep then starts only after the previous one has passed every tile plane.
//
// Two other schedules live here as well: the pencil schedule (k_gsp, one warp
// per 8 x 4 x-lines, neighbour lines exchanged by warp shuffles, per-pencil
// progress counts; pipelined batches on 3-D constant-coefficient operators)
// and, for small 1-/2-D grids, one block sweeping the whole iterate in shared
// memory along anti-diagonals (k_gs2d).  All three apply the same two-part
// update to every node (gs_old, then gs_new).
#include <cooperative_groups.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "hs_internal.h"

namespace hs {

template <int NDIM, int W>
struct GsTile;
// Tile shapes (one thread per x-line: TY * TZ threads per block), 3-D:
//   W = 0, 32 x 8 x 8 (two warps), for batches of four or more sweeps of one
//     direction, which pipeline: many small tiles keep more blocks resident
//     per SM (256^3, 200 sweeps: 325 us/sweep against 336 for 32 x 16 x 16,
//     341 for 32 x 16 x 8 and 32 x 8 x 16, 356 for 32 x 4 x 16);
//   W = 1, 32 x 16 x 16 (eight warps), for single sweeps and the symmetric
//     method, whose time is the number of tile planes times the time of a
//     tile (256^3 symmetric, residual every iteration: 3.48 ms/iteration
//     against 4.68 for 32 x 8 x 8).
// The W = 0 shape can be overridden at build time for measurements
// (-DHS_GS_TY=.. -DHS_GS_TZ=..).  2-D grids use 32 x 128 lines for both.
#ifndef HS_GS_TY
#define HS_GS_TY 8
#endif
#ifndef HS_GS_TZ
#define HS_GS_TZ 8
#endif
template <>
struct GsTile<3, 0> {
  static constexpr int TX = 32, TY = HS_GS_TY, TZ = HS_GS_TZ;
};
template <>
struct GsTile<3, 1> {
  static constexpr int TX = 32, TY = 16, TZ = 16;
};
template <int W>
struct GsTile<2, W> {
  static constexpr int TX = 32, TY = 128, TZ = 1;
};
template <int NDIM, int W>
constexpr int gs_threads() { return GsTile<NDIM, W>::TY * GsTile<NDIM, W>::TZ; }

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

// One tile of one sweep: load tile + halo, wavefront in shared memory, store.
template <typename T, int OPK, int NDIM, int W>
__device__ __forceinline__ void gs_tile(const GsArgs<T>& a, T* sm, int tile, bool backward) {
  constexpr int TX = GsTile<NDIM, W>::TX, TY = GsTile<NDIM, W>::TY, TZ = GsTile<NDIM, W>::TZ;
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
        if (gi >= 0 && gi < g.nx && gj >= 0 && gj < g.ny && gk >= 0 && gk < g.nz &&
            HS_IN_BOUNDS((long long)gk * g.plane + (long long)gj * g.nx + gi, g.N))
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
  // right-hand sides of the line's next four nodes in flight (a substep is
  // far shorter than a global load, so a one-substep prefetch would stall
  // every substep on it)
  T bq[4];
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const int ilq = HS_IL_AT(q + 1);
    bq[q] = ilq >= 0 ? __ldcg(bsrc + gbase + ilq) : T(0);
  }
  for (int s = 0; s < nsteps; s++) {
    const int il_n = HS_IL_AT(s + 1);
    const T bnext = bq[0];
    {
      const int il_f = HS_IL_AT(s + 5);
      bq[0] = bq[1];
      bq[1] = bq[2];
      bq[2] = bq[3];
      bq[3] = il_f >= 0 ? __ldcg(bsrc + gbase + il_f) : T(0);
    }
    OpRaw<T, OPK> onext{};
    if (il_n >= 0) onext = op_fetch<T, OPK, NDIM>(a.cf, g, gbase + il_n, i0 + il_n, gj, gk);
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
    if (gi < g.nx && gj2 < g.ny && gk2 < g.nz && HS_IN_BOUNDS((long long)gk2 * g.plane + (long long)gj2 * g.nx + gi, g.N))
      a.x[(long long)gk2 * g.plane + (long long)gj2 * g.nx + gi] = sm[((kk + ZOFF) * SY + (jj + 1)) * SX + ii + 1];
  }
  __syncthreads();
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

// Dataflow form of a batch: nsw sweeps (directions by `mode`; symmetric
// alternates forward and backward) with no grid-wide step.  Work items are
// (sweep, tile) pairs, taken from a counter in the order of the grid-step
// schedule: sweep t's tile plane S sits at step off(t) + S, with off(t) =
// 2t when all sweeps run one way (sweep t+1 trails sweep t by two tile
// planes) and t P when they alternate.  Before a tile is swept, warp 0 waits
// until its new-side face neighbours (lower ones for a forward sweep) have
// completed this sweep, and the tile itself and its old-side neighbours the
// previous one; after the tile is stored its sweep count is published.
// Every wait is on an item that comes earlier in the order, so the earliest
// unfinished item can always proceed.  `gsweep` (sweeps completed) and
// `cbase` (claims made) are the same in every block; each block ends a batch
// with exactly one claim past its end, so a batch takes nitems + G claims.
// Batches must be separated by a grid barrier.
template <typename T, int OPK, int NDIM, int W>
__device__ bool gs_batch_df(const GsArgs<T>& a, T* sm, int nsw, int mode, unsigned& gsweep,
                            unsigned long long& cbase) {
  __shared__ long long s_item;
  __shared__ int s_tile, s_bw, s_ok;
  const int nt = a.ntx * a.nty * a.ntz;
  const int P = a.P;
  const int L = mode == HS_GS_SYMMETRIC ? P : 2;
  const long long nitems = (long long)nsw * nt;
  // lane 0 of warp 0: position of the schedule (its claims only grow)
  int tau_c = 0;
  long long cum_c = 0;   // items before step tau_c
  while (true) {
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      long long u = 0;
      int tile = 0, t = 0, bw = 0;
      if (lane == 0) {
        u = (long long)(atomicAdd(a.claim, 1ull) - cbase);
        if (u < nitems) {
          while (true) {
            const int t_lo = tau_c < P ? 0 : (tau_c - P) / L + 1;
            const int t_hi = min(nsw - 1, tau_c / L);
            long long rem = u - cum_c;
            int found = -1;
            for (int tt = t_lo; tt <= t_hi; tt++) {
              const int S = tau_c - L * tt;
              const bool b2 = mode == HS_GS_BACKWARD || (mode == HS_GS_SYMMETRIC && (tt & 1));
              const int Se = b2 ? P - 1 - S : S;
              const int cnt = a.plane_off[Se + 1] - a.plane_off[Se];
              if (rem < cnt) {
                found = tt;
                tile = a.plane_tiles[a.plane_off[Se] + (int)rem];
                bw = b2;
                break;
              }
              rem -= cnt;
            }
            if (found >= 0) {
              t = found;
              break;
            }
            cum_c = u - rem;   // all items of step tau_c lie before u
            tau_c++;
          }
        }
      }
      u = __shfl_sync(0xffffffffu, u, 0);
      tile = __shfl_sync(0xffffffffu, tile, 0);
      t = __shfl_sync(0xffffffffu, t, 0);
      bw = __shfl_sync(0xffffffffu, bw, 0);
      int ok = 1;
      if (u < nitems) {
        const unsigned gs = gsweep + (unsigned)t;
        const int I = tile % a.ntx, J = (tile / a.ntx) % a.nty, K = tile / (a.ntx * a.nty);
        // lane 0: the tile itself; lanes 1..6: -x, +x, -y, +y, -z, +z
        const unsigned* f = nullptr;
        unsigned target = 0;
        if (lane == 0) {
          f = a.tile_done + tile;
          target = gs;
        } else if (lane <= 6) {
          const int d = (lane - 1) >> 1, up = (lane - 1) & 1;
          const int step = up ? 1 : -1;
          const int c = d == 0 ? I + step : (d == 1 ? J + step : K + step);
          const int lim = d == 0 ? a.ntx : (d == 1 ? a.nty : a.ntz);
          if (c >= 0 && c < lim) {
            f = a.tile_done + tile + step * (d == 0 ? 1 : (d == 1 ? a.ntx : a.ntx * a.nty));
            const bool newside = bw ? up : !up;
            target = newside ? gs + 1 : gs;
          }
        }
        ok = gs_poll(f != nullptr, f, target, a.cm.ctrl);
      }
      if (lane == 0) {
        s_item = u;
        s_tile = tile;
        s_bw = bw;
        s_ok = ok;
        if (u < nitems) s_item = (long long)t;   // the sweep, for the publish below
        else s_item = -1;
      }
    }
    __syncthreads();
    const long long t = s_item;
    if (!s_ok) return false;
    if (t < 0) break;
    const int tile = s_tile;
    gs_tile<T, OPK, NDIM, W>(a, sm, tile, s_bw != 0);   // ends with a block barrier
    if (threadIdx.x == 0) {
      __threadfence();
      st_release(a.tile_done + tile, gsweep + (unsigned)t + 1u);
    }
  }
  gsweep += (unsigned)nsw;
  cbase += (unsigned long long)nitems + gridDim.x;
  return true;
}

template <typename T, int OPK, int NDIM, int W>
__global__ void __launch_bounds__(gs_threads<NDIM, W>()) k_gs(GsArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  // the reductions run between batches, when no tile is staged: their
  // scratch shares the tile buffer, which keeps a 32 x 8 x 8 FP64 block at
  // 28.2 KB of shared memory (eight resident blocks per SM instead of seven)
  static_assert((GsTile<NDIM, W>::TX + 2) * (GsTile<NDIM, W>::TY + 2) * (NDIM == 3 ? GsTile<NDIM, W>::TZ + 2 : 1) *
                        sizeof(T) >= 32 * MAX_SCAL * sizeof(double),
                "the tile buffer must hold the reduction scratch");
  double* sh = reinterpret_cast<double*>(smraw);
  const long long N = a.g.N;

  double acc[1] = {0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    T bv = a.b[i];
    if (OPK != OP_VARK) a.bD[i] = bv * a.invd;
    acc[0] += widen(bv) * widen(bv);
  }
  // schedule state, ordered before its first use by the reduction below
  const int ntiles = a.ntx * a.nty * a.ntz;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x) a.tile_done[t] = 0u;
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.claim = 0ull;
  unsigned gsweep = 0;
  unsigned long long cbase = 0;
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
      if (!gs_batch_df<T, OPK, NDIM, W>(a, sm, a.mode == HS_GS_SYMMETRIC ? 2 * nb : nb, a.mode, gsweep, cbase))
        return;
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
// Pencil schedule (3-D, constant coefficients).  A warp owns a pencil of
// GSP_PY x GSP_PZ x-lines, lane l = jl + GSP_PY kl on line (j, k) =
// (J GSP_PY + jl, K GSP_PZ + kl), and streams along x two nodes (a pair) per
// substep: in the sweep's frame (mirrored for a backward sweep) lane
// (jm, km) handles pair u - D at substep u, D = jm + km.  The lexicographic
// order holds node by node:
//   * the x neighbours are the lane's own: the new one is the second node of
//     its previous pair, the old ones come from its line in memory;
//   * the new-side y and z neighbours (j - 1, k - 1 in a forward sweep) are
//     the pair the neighbouring lanes computed at the previous substep
//     (shuffled up by 1 and GSP_PY lanes), the old-side ones the old pair the
//     lanes on the other side handle next (shuffled down);
//   * lines of other pencils (lanes on the pencil's faces) come from memory,
//     GSP_PF pairs ahead, after waiting until the new-side pencils have
//     published enough pairs of this sweep and the old-side pencils enough of
//     the previous sweep (all of it when the direction flips).
// A warp publishes, every GSP_CH substeps, how many pairs all its lanes have
// stored (per-pencil count, monotonic over sweeps: sweep t, P pairs ->
// t NQ + P).  Pencils are dealt to warps statically in consecutive runs and
// each warp takes its pencils sweep by sweep in the sweep's direction, so the
// earliest unfinished (sweep, pencil) item only ever waits on finished items:
// no deadlock.  Sweeps overlap (a pencil starts sweep t + 1 while pencils
// above it are still in sweep t) when every warp owns one pencil; the
// automatic choice takes this schedule only then.  No block barrier inside
// a sweep: each warp runs on its own.  The update arithmetic is that of
// gs_tile (gs_old then gs_new), so iterates are bitwise those of the tile
// schedule.
// ---------------------------------------------------------------------------

constexpr int GSP_PY = 8, GSP_PZ = 4;   // lines per pencil (one warp)
#ifndef HS_GSP_CH
#define HS_GSP_CH 18
#endif
constexpr int GSP_CH = HS_GSP_CH;       // substeps between progress updates
constexpr int GSP_PF = 2;               // pencil-face pairs loaded ahead
constexpr int GSP_WARPS = 4;            // warps per block
constexpr int GSP_DMAX = (GSP_PY - 1) + (GSP_PZ - 1);

struct GspArgs {
  unsigned* prog;   // per pencil: pairs stored, t NQ + P
  void* zero;       // 64 bytes of zeros (read in place of values outside the grid)
  int nJ, nK, NP, NQ;
};

template <typename T>
struct GPair {
  T a, b;   // sweep order: a first
};

template <typename T>
struct Vec2;
template <>
struct Vec2<double> {
  using type = double2;
};
template <>
struct Vec2<float> {
  using type = float2;
};

// Pair qq (sweep frame) of the line starting at element `line` of arr:
// positions 2q, 2q + 1 with q = qq (forward) or NQ - 1 - qq (backward, a =
// 2q + 1 first).  Outside the line (line < 0 for no line, qq outside
// [0, NQ), the half pair past an odd n_x) the value is read from `zero`, a
// few zero words in the workspace, rather than selected afterwards: a select
// on a loaded value would wait for the load at once and undo the prefetch.
template <typename T, bool BW, bool VEC>
__device__ __forceinline__ GPair<T> gsp_load(const T* arr, long long line, int qq, int NQ, int nx, long long N,
                                              const T* zero) {
  const int q = BW ? NQ - 1 - qq : qq;
  const long long e = line + 2 * q;
  const bool in = line >= 0 && qq >= 0 && qq < NQ && HS_IN_BOUNDS(e, N);
  T lo, hi;
  if constexpr (VEC) {
    const typename Vec2<T>::type v = __ldcg(reinterpret_cast<const typename Vec2<T>::type*>(in ? arr + e : zero));
    lo = v.x;
    hi = v.y;
  } else {
    const bool in_hi = in && 2 * q + 1 < nx && HS_IN_BOUNDS(e + 1, N);
    lo = __ldcg(in ? arr + e : zero);
    hi = __ldcg(in_hi ? arr + e + 1 : zero);
  }
  GPair<T> r;
  r.a = BW ? hi : lo;
  r.b = BW ? lo : hi;
  return r;
}

template <typename T, bool BW, bool VEC>
__device__ __forceinline__ void gsp_store(T* arr, long long line, int qq, int NQ, int nx, long long N, T na, T nb) {
  const int q = BW ? NQ - 1 - qq : qq;
  const long long e = line + 2 * q;
  const bool has_hi = 2 * q + 1 < nx;
  if (!HS_IN_BOUNDS(e, N) || (has_hi && !HS_IN_BOUNDS(e + 1, N))) return;
  const T lo = BW ? nb : na, hi = BW ? na : nb;
  if constexpr (VEC) {
    typename Vec2<T>::type v;
    v.x = lo;
    v.y = hi;
    *reinterpret_cast<typename Vec2<T>::type*>(arr + e) = v;
  } else {
    arr[e] = lo;
    if (has_hi) arr[e + 1] = hi;
  }
}

// The polling lanes (mine) wait until *f >= target, bounded by the solve's
// timeout; all 32 lanes call it and leave together.
__device__ __forceinline__ bool gsp_poll(bool mine, const unsigned* f, unsigned target, Ctrl* ctrl) {
  return gs_poll(mine, f, target, ctrl);
}

template <typename T, int OPK, bool BW, bool VEC>
__device__ bool gsp_item(const GsArgs<T>& a, const GspArgs& G, int p, unsigned tq, bool has_prev, bool same_dir) {
  const Geom& g = a.g;
  const int lane = threadIdx.x & 31;
  const int jl = lane % GSP_PY, kl = lane / GSP_PY;
  const int jm = BW ? GSP_PY - 1 - jl : jl, km = BW ? GSP_PZ - 1 - kl : kl;
  const int D = jm + km;
  const int J = p % G.nJ, K = p / G.nJ;
  const int j = J * GSP_PY + jl, k = K * GSP_PZ + kl;
  const bool valid = j < g.ny && k < g.nz;
  const int s = BW ? 1 : -1;   // towards the new side
  const int nx = g.nx, NQ = G.NQ;
  const T* zero = reinterpret_cast<const T*>(G.zero);
  const T* bsrc = a.bD;
  T* x = a.x;
  const long long N = g.N;
  const long long line = valid ? (long long)k * g.plane + (long long)j * nx : -1;
  // the pencil-face lines this lane reads (-1: outside the grid, zeros)
  const bool fny = jm == 0, fnz = km == 0, foy = jm == GSP_PY - 1, foz = km == GSP_PZ - 1;
  const long long lfy = (valid && fny && j + s >= 0 && j + s < g.ny)   ? line + (long long)s * nx
                        : (valid && foy && j - s >= 0 && j - s < g.ny) ? line - (long long)s * nx
                                                                       : -1;
  const long long lfz = (valid && fnz && k + s >= 0 && k + s < g.nz)   ? line + (long long)s * g.plane
                        : (valid && foz && k - s >= 0 && k - s < g.nz) ? line - (long long)s * g.plane
                                                                       : -1;
  // neighbouring pencils: new side (J + s, K), (J, K + s); old side (J - s, K), (J, K - s)
  const int pny = (J + s >= 0 && J + s < G.nJ) ? p + s : -1;
  const int pnz = (K + s >= 0 && K + s < G.nK) ? p + s * G.nJ : -1;
  const int poy = (J - s >= 0 && J - s < G.nJ) ? p - s : -1;
  const int poz = (K - s >= 0 && K - s < G.nK) ? p - s * G.nJ : -1;
  // lanes 0..3 poll one neighbour each
  const int pw = lane == 0 ? pny : (lane == 1 ? pnz : (lane == 2 ? poy : (lane == 3 ? poz : -1)));
  const bool pw_new = lane < 2;
  const bool pw_on = pw >= 0 && (pw_new || has_prev);

  // Queue slots: old values of the lane's own line for pairs qq, qq + 1,
  // qq + 2 (three slots; a substep uses the first two and refills the first
  // with qq + 3), b / a_ii and the pencil-face lines for pairs qq, qq + 1 (two
  // slots, refilled with qq + 2).  The substep loop is unrolled six times with
  // the slots' roles rotated, so no register is copied while its load is in
  // flight.
  struct Faces {
    GPair<T> y, z;
  };
  GPair<T> o0, o1, o2, b0, b1;
  Faces f0, f1;
  GPair<T> last{T(0), T(0)};   // new values of the previous pair
  static_assert(GSP_PY > 1 && GSP_PZ > 1, "pencil faces must be distinct lanes");
  static_assert(GSP_CH % 6 == 0, "chunks hold whole rotations of the queue slots");
  const OpRaw<T, OPK> onone{};
  auto fill_f = [&](Faces& f, int qq) {
    f.y = gsp_load<T, BW, VEC>(x, lfy, qq, NQ, nx, N, zero);
    f.z = gsp_load<T, BW, VEC>(x, lfz, qq, NQ, nx, N, zero);
  };
  // one substep: oc / on = own old pairs qq / qq + 1, bc = b of pair qq,
  // fc = face lines at pair qq; refills oc with qq + 3, bc and fc with qq + 2
  auto step = [&](int u, GPair<T>& oc, const GPair<T>& on, GPair<T>& bc, Faces& fc) {
    const int qq = u - D;
    // neighbour lines inside the pencil: new side = the pair the lanes one
    // line towards the new side computed last substep, old side = the old
    // pair the lanes on the other side handle next
    GPair<T> ny, nz, oy, oz;
    if constexpr (!BW) {
      ny.a = __shfl_up_sync(0xffffffffu, last.a, 1);
      ny.b = __shfl_up_sync(0xffffffffu, last.b, 1);
      nz.a = __shfl_up_sync(0xffffffffu, last.a, GSP_PY);
      nz.b = __shfl_up_sync(0xffffffffu, last.b, GSP_PY);
      oy.a = __shfl_down_sync(0xffffffffu, on.a, 1);
      oy.b = __shfl_down_sync(0xffffffffu, on.b, 1);
      oz.a = __shfl_down_sync(0xffffffffu, on.a, GSP_PY);
      oz.b = __shfl_down_sync(0xffffffffu, on.b, GSP_PY);
    } else {
      ny.a = __shfl_down_sync(0xffffffffu, last.a, 1);
      ny.b = __shfl_down_sync(0xffffffffu, last.b, 1);
      nz.a = __shfl_down_sync(0xffffffffu, last.a, GSP_PY);
      nz.b = __shfl_down_sync(0xffffffffu, last.b, GSP_PY);
      oy.a = __shfl_up_sync(0xffffffffu, on.a, 1);
      oy.b = __shfl_up_sync(0xffffffffu, on.b, 1);
      oz.a = __shfl_up_sync(0xffffffffu, on.a, GSP_PY);
      oz.b = __shfl_up_sync(0xffffffffu, on.b, GSP_PY);
    }
    // lanes on the pencil's faces take those lines from memory
    ny.a = fny ? fc.y.a : ny.a;
    ny.b = fny ? fc.y.b : ny.b;
    oy.a = foy ? fc.y.a : oy.a;
    oy.b = foy ? fc.y.b : oy.b;
    nz.a = fnz ? fc.z.a : nz.a;
    nz.b = fnz ? fc.z.b : nz.b;
    oz.a = foz ? fc.z.a : oz.a;
    oz.b = foz ? fc.z.b : oz.b;
    if (valid && qq >= 0 && qq < NQ) {
      const int q = BW ? NQ - 1 - qq : qq;
      const bool va = BW ? (2 * q + 1 < nx) : true;
      const bool vb = BW ? true : (2 * q + 1 < nx);
      T na = T(0), nb = T(0);
      if (va) {
        const T y = gs_old<T, OPK, 3>(a.cf, onone, bc.a, oc.b, oy.a, oz.a, BW);
        na = gs_new<T, OPK, 3>(a.cf, onone, y, last.b, ny.a, nz.a, BW);
      }
      if (vb) {
        const T y = gs_old<T, OPK, 3>(a.cf, onone, bc.b, on.a, oy.b, oz.b, BW);
        nb = gs_new<T, OPK, 3>(a.cf, onone, y, na, ny.b, nz.b, BW);
      }
      gsp_store<T, BW, VEC>(x, line, qq, NQ, nx, N, na, nb);
      last.a = na;
      last.b = nb;
    }
    oc = gsp_load<T, BW, VEC>(x, line, qq + 3, NQ, nx, N, zero);
    bc = gsp_load<T, BW, VEC>(bsrc, line, qq + 2, NQ, nx, N, zero);
    fill_f(fc, qq + GSP_PF);
  };
  const int NU = NQ + GSP_DMAX;
  for (int u0 = 0; u0 < NU; u0 += GSP_CH) {
    // wait until the faces this chunk loads are final
    {
      const int c = u0 / GSP_CH;
      const unsigned need = (unsigned)min(NQ, (c + 1) * GSP_CH + GSP_PF);
      unsigned target = 0;
      if (pw_new) target = tq + need;
      else target = same_dir ? tq - (unsigned)NQ + need : tq;
      if (!gsp_poll(pw_on, pw_on ? G.prog + pw : nullptr, target, a.cm.ctrl)) return false;
    }
    if (u0 == 0) {
      o0 = gsp_load<T, BW, VEC>(x, line, -D, NQ, nx, N, zero);
      o1 = gsp_load<T, BW, VEC>(x, line, -D + 1, NQ, nx, N, zero);
      o2 = gsp_load<T, BW, VEC>(x, line, -D + 2, NQ, nx, N, zero);
      b0 = gsp_load<T, BW, VEC>(bsrc, line, -D, NQ, nx, N, zero);
      b1 = gsp_load<T, BW, VEC>(bsrc, line, -D + 1, NQ, nx, N, zero);
      fill_f(f0, -D);
      fill_f(f1, -D + 1);
    }
    const int u1 = min(u0 + GSP_CH, NU);
    for (int u = u0; u < u1; u += 6) {
      step(u, o0, o1, b0, f0);
      if (u + 1 < u1) step(u + 1, o1, o2, b1, f1);
      if (u + 2 < u1) step(u + 2, o2, o0, b0, f0);
      if (u + 3 < u1) step(u + 3, o0, o1, b1, f1);
      if (u + 4 < u1) step(u + 4, o1, o2, b0, f0);
      if (u + 5 < u1) step(u + 5, o2, o0, b1, f1);
    }
    // publish the pairs every lane has stored
    __syncwarp();
    if (lane == 0) {
      __threadfence();
      st_relaxed(G.prog + p, tq + (unsigned)max(0, min(NQ, u1 - GSP_DMAX)));
    }
  }
  return true;
}

// nsw sweeps (directions by mode) over every pencil.  gsweep: sweeps done
// before this batch, the same in every warp.
template <typename T, int OPK, bool VEC>
__device__ bool gsp_batch(const GsArgs<T>& a, const GspArgs& G, int nsw, int mode, unsigned& gsweep) {
  const int W = gridDim.x * GSP_WARPS;
  const int w = blockIdx.x * GSP_WARPS + (threadIdx.x >> 5);
  auto dir_bw = [&](unsigned tg) {
    return mode == HS_GS_BACKWARD || (mode == HS_GS_SYMMETRIC && (tg & 1u));
  };
  // a warp owns consecutive pencils (neighbours in x-lines' j order, so
  // that a second pencil waits on the first rather than on a far one)
  const int per = (G.NP + W - 1) / W;
  const int p0 = w * per, p1 = min(G.NP, p0 + per);
  if (p0 < p1) {
    const int nmine = p1 - p0;
    for (int t = 0; t < nsw; t++) {
      const unsigned tg = gsweep + (unsigned)t;
      const bool bw = dir_bw(tg);
      const bool has_prev = tg > 0;
      const bool same_dir = has_prev && dir_bw(tg - 1) == bw;
      const unsigned tq = tg * (unsigned)G.NQ;
      for (int m = 0; m < nmine; m++) {
        const int p = p0 + (bw ? nmine - 1 - m : m);
        const bool ok = bw ? gsp_item<T, OPK, true, VEC>(a, G, p, tq, has_prev, same_dir)
                           : gsp_item<T, OPK, false, VEC>(a, G, p, tq, has_prev, same_dir);
        if (!ok) return false;
      }
    }
  }
  gsweep += (unsigned)nsw;
  return true;
}

// Four blocks of four warps per SM (128 registers a thread): all 2048
// pencils of a 256^3 grid resident at once.
#ifndef HS_GSP_MINB
#define HS_GSP_MINB 4
#endif
template <typename T, int OPK, bool VEC>
__global__ void __launch_bounds__(32 * GSP_WARPS, HS_GSP_MINB) k_gsp(GsArgs<T> a, GspArgs G) {
  __shared__ double sh[32 * MAX_SCAL];
  const long long N = a.g.N;
  double acc[1] = {0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    T bv = a.b[i];
    a.bD[i] = bv * a.invd;
    acc[0] += widen(bv) * widen(bv);
  }
  // progress counts, ordered before their first use by the reduction below
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < G.NP; q += gridDim.x * blockDim.x) G.prog[q] = 0u;
  if (blockIdx.x == 0 && threadIdx.x < 16) reinterpret_cast<unsigned*>(G.zero)[threadIdx.x] = 0u;
  unsigned gsweep = 0;
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
    if (!gs_residual<T, OPK, 3>(a, nullptr, sh, bb[0], &rel)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.cm.hist[0] = rel;
    if (!(rel > a.tol)) status = isfinite(rel) ? DS_CONVERGED : DS_NONFINITE;
    else status = DS_MAXIT;
  }
  if (!(a.tol > 0.0) || status == DS_MAXIT) {
    while (done < a.maxit) {
      int nb = (a.tol > 0.0) ? min(a.check_every, a.maxit - done) : a.maxit - done;
      if (!gsp_batch<T, OPK, VEC>(a, G, a.mode == HS_GS_SYMMETRIC ? 2 * nb : nb, a.mode, gsweep)) return;
      done += nb;
      if (a.tol > 0.0) {
        if (!gs_residual<T, OPK, 3>(a, nullptr, sh, bb[0], &rel)) return;
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
// Small 2-D (and 1-D) grids: one block holds the whole iterate in shared
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
// The update arithmetic is that of gs_tile (gs_old then gs_new).
// ---------------------------------------------------------------------------

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

template <int NDIM, int W>
static void tile_counts(const hs_op* A, int* ntx, int* nty, int* ntz) {
  *ntx = (int)((A->n[0] + GsTile<NDIM, W>::TX - 1) / GsTile<NDIM, W>::TX);
  *nty = (int)((A->n[1] + GsTile<NDIM, W>::TY - 1) / GsTile<NDIM, W>::TY);
  *ntz = (int)((A->n[2] + GsTile<NDIM, W>::TZ - 1) / GsTile<NDIM, W>::TZ);
}

// Tile-plane tables on the device: off[S] = number of tiles on planes below S
// (S = I + J + K; off[P] = all tiles), then the tile ids of each plane in
// increasing id order.  With a x b x c tiles, the tiles (I, J) of one z layer
// on plane u number
//   N2(u) = max(0, min(u, a - 1) - max(0, u - b + 1) + 1)   (u >= 0),
// a plane's tiles sum N2 over the layers, and a tile's rank inside its plane
// counts the layers below it and the rows J' < J of its own layer that reach
// the plane.  Computed on the device (no host staging), so a solve can be
// captured in a CUDA graph.
__device__ __forceinline__ int gs_n2(int u, int a, int b) {
  if (u < 0) return 0;
  const int lo = u - b + 1 > 0 ? u - b + 1 : 0;
  const int hi = u < a - 1 ? u : a - 1;
  return hi >= lo ? hi - lo + 1 : 0;
}

__global__ void k_gs_plane_off(int a, int b, int c, int P, int* off) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q <= P; q += gridDim.x * blockDim.x) {
    int sum = 0;
    for (int sp = 0; sp < q; sp++)
      for (int k = 0; k < c; k++) sum += gs_n2(sp - k, a, b);
    off[q] = sum;
  }
}

__global__ void k_gs_plane_tiles(int a, int b, int c, const int* off, int* tiles) {
  const int nt = a * b * c;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
    const int I = t % a, J = (t / a) % b, K = t / (a * b);
    const int S = I + J + K;
    int rank = 0;
    for (int k = 0; k < K; k++) rank += gs_n2(S - k, a, b);
    for (int j = 0; j < J; j++) {
      const int i = S - K - j;
      rank += (i >= 0 && i < a) ? 1 : 0;
    }
    tiles[off[S] + rank] = t;
  }
}

// Tile count and tile planes of the larger table (the W = 0 shape has the
// smaller tiles in every direction).
static void gs_counts(const hs_op* A, int* ntiles, int* P) {
  static_assert(GsTile<3, 0>::TY <= GsTile<3, 1>::TY && GsTile<3, 0>::TZ <= GsTile<3, 1>::TZ,
                "workspace sizing assumes the W = 0 tiles are the smaller ones");
  int a, b, c;
  if (A->ndim >= 3) tile_counts<3, 0>(A, &a, &b, &c);
  else tile_counts<2, 0>(A, &a, &b, &c);
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
  // b / a_ii, the tile-plane tables, per-tile sweep counts, the claim
  // counter, then the pencil schedule's per-pencil progress counts
  const size_t npen = (size_t)((A->n[1] + GSP_PY - 1) / GSP_PY) * (size_t)((A->n[2] + GSP_PZ - 1) / GSP_PZ);
  return ((N * es + 255) & ~(size_t)255) + ((ints * 4 + 255) & ~(size_t)255) + (((size_t)nt * 4 + 255) & ~(size_t)255) +
         256 + ((npen * 4 + 255) & ~(size_t)255) + 256;
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

template <typename T, int OPK, int NDIM, int W>
static hs_status gs_run_t(const SolveArgs& sa, hs_result* res, double* hist) {
  constexpr int TX = GsTile<NDIM, W>::TX, TY = GsTile<NDIM, W>::TY, TZ = GsTile<NDIM, W>::TZ;
  constexpr int THREADS = TY * TZ;
  static_assert(THREADS % 32 == 0 && THREADS <= 1024, "GS tiles use whole warps of lines");
  const hs_op* A = sa.A;
  Geom g = geom_of(A);
  Carve c{sa.ws, 0, sa.ws_bytes, true};
  Common cm = carve_common(c, sa.maxit);
  GsArgs<T> a = {};
  a.bD = c.take<T>(g.N);
  int ntx, nty, ntz;
  tile_counts<NDIM, W>(A, &ntx, &nty, &ntz);
  if (NDIM == 2) ntz = 1;
  const int ntiles = ntx * nty * ntz, P = ntx + nty + ntz - 2;
  int* tabs = c.take<int>((size_t)ntiles + P + 1);
  a.tile_done = c.take<unsigned>((size_t)ntiles);
  a.claim = c.take<unsigned long long>(1);
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
  // tile planes: offsets then tile ids grouped by I + J + K (device kernels)
  k_gs_plane_off<<<(P + 1 + 127) / 128, 128, 0, sa.stream>>>(ntx, nty, ntz, P, tabs);
  k_gs_plane_tiles<<<(ntiles + 255) / 256, 256, 0, sa.stream>>>(ntx, nty, ntz, tabs, tabs + P + 1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "tile tables");
  {
    hs_status si = init_ctrl(cm, sa.o, sa.stream);
    if (si != HS_OK) return si;
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
  auto kern = k_gs<T, OPK, NDIM, W>;
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
  if (sa.o.max_blocks > 0) grid = std::min(grid, sa.o.max_blocks);
  void* args[] = {&a};
  e = cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(THREADS), args, smem, sa.stream);
  if (e != cudaSuccess) return cuda_fail(e, "cooperative launch");
  if (OPK == OP_VARK && sa.o.true_residual) {
    hs_status s = setup_vark(A, sa.dtype, D, ax, ay, az, false, sa.stream);
    if (s != HS_OK) return s;
  }
  hs_status sd = hs_dbg_take(sa.stream);
  if (sd != HS_OK) return sd;
  return finish_solve_pub(sa, cm, D, ax, ay, az, a.bD, res, hist, sa.tol > 0.0);
}

// The pencil schedule applies to 3-D constant-coefficient operators whose
// progress counts (sweeps x pairs per line) fit in 32 bits.
static bool gsp_applies(const hs_op* A, const SolveArgs& sa) {
  if (A->ndim != 3) return false;
  const int opk = opkind_of(A);
  if (opk != OP_SYM && opk != OP_NONSYM) return false;
  const long long nq = (A->n[0] + 1) / 2;
  const long long sweeps = (long long)sa.maxit * (sa.o.gs_mode == HS_GS_SYMMETRIC ? 2 : 1) + 2;
  return sweeps * nq < (1ll << 31);
}

// Every pencil gets a warp of its own (so that sweeps overlap), and there
// are enough of them to keep at least twelve warps busy on every SM (with
// fewer, the FP64 pipe idles behind each warp's dependent chain: 192^3 runs
// 153 us per sweep against 142 with tiles)?
template <typename T, int OPK>
static bool gsp_fits(const hs_op* A, const hs_opts& o) {
  const long long np = ((A->n[1] + GSP_PY - 1) / GSP_PY) * ((A->n[2] + GSP_PZ - 1) / GSP_PZ);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gsp<T, OPK, true>, 32 * GSP_WARPS, 0) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  long long blocks = std::min<long long>((long long)per_sm * sm_count(), MAX_BLOCKS);
  if (o.max_blocks > 0) blocks = std::min<long long>(blocks, o.max_blocks);
  return np <= blocks * GSP_WARPS && np >= 12ll * sm_count();
}

template <typename T, int OPK>
static hs_status gsp_run_t(const SolveArgs& sa, hs_result* res, double* hist) {
  const hs_op* A = sa.A;
  Geom g = geom_of(A);
  Carve c{sa.ws, 0, sa.ws_bytes, true};
  Common cm = carve_common(c, sa.maxit);
  GsArgs<T> a = {};
  a.bD = c.take<T>(g.N);
  GspArgs G = {};
  G.nJ = (int)((g.ny + GSP_PY - 1) / GSP_PY);
  G.nK = (int)((g.nz + GSP_PZ - 1) / GSP_PZ);
  G.NP = G.nJ * G.nK;
  G.NQ = (int)((g.nx + 1) / 2);
  G.prog = c.take<unsigned>((size_t)G.NP);
  G.zero = c.take<unsigned>(16);
  if (!c.ok) {
    set_error("workspace too small for Gauss-Seidel");
    return HS_ERR_WORKSPACE;
  }
  // pairs load as aligned vectors when every line starts on a pair boundary
  const size_t vb = 2 * sizeof(T);
  const bool vec = g.nx % 2 == 0 && ((uintptr_t)sa.x % vb) == 0 && ((uintptr_t)a.bD % vb) == 0;
  {
    hs_status si = init_ctrl(cm, sa.o, sa.stream);
    if (si != HS_OK) return si;
  }
  a.cf = gs_jacobi_coef<T>(A, &a.invd, &a.dscale2);
  a.g = g;
  a.b = (const T*)sa.b;
  a.x = (T*)sa.x;
  a.cm = cm;
  a.maxit = sa.maxit;
  a.mode = sa.o.gs_mode;
  a.check_every = sa.o.check_every;
  a.tol = sa.tol;
  auto kern = vec ? k_gsp<T, OPK, true> : k_gsp<T, OPK, false>;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * GSP_WARPS, 0);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
  if (per_sm < 1) {
    set_error("Gauss-Seidel kernel cannot be resident");
    return HS_ERR_CUDA;
  }
  int grid = std::min(per_sm * sm_count(), MAX_BLOCKS);
  grid = std::min(grid, (G.NP + GSP_WARPS - 1) / GSP_WARPS);
  if (sa.o.max_blocks > 0) grid = std::min(grid, sa.o.max_blocks);
  grid = std::max(grid, 1);
  void* args[] = {&a, &G};
  e = cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(32 * GSP_WARPS), args, 0, sa.stream);
  if (e != cudaSuccess) return cuda_fail(e, "cooperative launch");
  hs_status sd = hs_dbg_take(sa.stream);
  if (sd != HS_OK) return sd;
  return finish_solve_pub(sa, cm, nullptr, nullptr, nullptr, nullptr, a.bD, res, hist, sa.tol > 0.0);
}

// Largest iterate the single-block 2-D path holds in shared memory.
constexpr size_t GS2D_SMEM_MAX = 200 * 1024;

template <typename T>
static bool gs2d_applies(const hs_op* A, const hs_opts& o) {
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
  if (OPK == OP_VARK) {
    // the workspace sizing reserves the tile tables first; the coefficient
    // arrays follow them in both layouts
    int nt, P;
    gs_counts(A, &nt, &P);
    c.take<int>((size_t)nt + P + 1);
    c.take<unsigned>((size_t)nt);
    c.take<unsigned long long>(1);
    D = c.take<T>(g.N);
    ax = c.take<T>(g.N);
    ay = c.take<T>(g.N);
    az = c.take<T>(g.N);
  }
  if (!c.ok) {
    set_error("workspace too small for Gauss-Seidel");
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
    a.cf = gs_jacobi_coef<T>(A, &a.invd, &a.dscale2);
  }
  a.g = g;
  a.b = (const T*)sa.b;
  a.x = (T*)sa.x;
  a.cm = cm;
  a.maxit = sa.maxit;
  a.mode = sa.o.gs_mode;
  a.check_every = sa.o.check_every;
  a.tol = sa.tol;
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
  if (OPK == OP_VARK && sa.o.true_residual) {
    s = setup_vark(A, sa.dtype, D, ax, ay, az, false, sa.stream);
    if (s != HS_OK) return s;
  }
  s = hs_dbg_take(sa.stream);
  if (s != HS_OK) return s;
  return finish_solve_pub(sa, cm, D, ax, ay, az, a.bD, res, hist, sa.tol > 0.0);
}

// The cluster form: 2-D grids of at least two rows per CTA whose rows fit the
// CTAs' shared memory, unless the caller caps the grid (max_blocks = 1: one
// block; more: the tile schedule).
template <typename T>
static bool gs2dc_applies(const hs_op* A, const hs_opts& o) {
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
  if (OPK == OP_VARK) {
    // the same layout as the other schedules: tile tables, then coefficients
    int nt, P;
    gs_counts(A, &nt, &P);
    c.take<int>((size_t)nt + P + 1);
    c.take<unsigned>((size_t)nt);
    c.take<unsigned long long>(1);
    D = c.take<T>(g.N);
    ax = c.take<T>(g.N);
    ay = c.take<T>(g.N);
    az = c.take<T>(g.N);
  }
  if (!c.ok) {
    set_error("workspace too small for Gauss-Seidel");
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
    a.cf = gs_jacobi_coef<T>(A, &a.invd, &a.dscale2);
  }
  a.g = g;
  a.b = (const T*)sa.b;
  a.x = (T*)sa.x;
  a.cm = cm;
  a.maxit = sa.maxit;
  a.mode = sa.o.gs_mode;
  a.check_every = sa.o.check_every;
  a.tol = sa.tol;
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
  if (OPK == OP_VARK && sa.o.true_residual) {
    s = setup_vark(A, sa.dtype, D, ax, ay, az, false, sa.stream);
    if (s != HS_OK) return s;
  }
  s = hs_dbg_take(sa.stream);
  if (s != HS_OK) return s;
  return finish_solve_pub(sa, cm, D, ax, ay, az, a.bD, res, hist, sa.tol > 0.0);
}

// Warp 0 waits for a sweep count that nothing publishes (diagnostic).
__global__ void k_diag_gs(Ctrl* ctrl, const unsigned* flag) {
  if (threadIdx.x < 32) gs_poll(threadIdx.x == 0, flag, 1u, ctrl);
}

hs_status diag_gs_wait(Ctrl* ctrl, const unsigned* flag, cudaStream_t st) {
  k_diag_gs<<<1, 32, 0, st>>>(ctrl, flag);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HS_OK : cuda_fail(e, "diagnostic launch");
}

hs_status run_gauss_seidel(const SolveArgs& sa, hs_result* res, double* hist) {
  const int opk = opkind_of(sa.A);
  const bool d3 = sa.A->ndim >= 3;
  if (opk == OP_BOX27) return run_gauss_seidel27(sa, res, hist);
  // batches of four or more sweeps of one direction pipeline (small tiles;
  // on small 2-D grids one cluster: 128^2, 5.6 against 19 us per sweep with
  // one block); single sweeps and symmetric batches are bound by the chain of
  // steps (large tiles, fewer planes; on small 2-D grids one block, whose
  // barrier is cheaper than the cluster's: 383 against 588 us per symmetric
  // iteration at 128^2)
  const int per_batch = sa.tol > 0.0 ? sa.o.check_every : sa.maxit;
  const bool deep = sa.o.gs_mode == HS_GS_SYMMETRIC || per_batch < 4;
  const bool pencils = gsp_applies(sa.A, sa);
  if (sa.o.gs_schedule == 2 && !pencils) {
    set_error("the pencil schedule needs a 3-D Laplacian or upwind operator");
    return HS_ERR_INVALID;
  }
  if (sa.o.gs_schedule == 3) {
    const bool fits = sa.dtype == HS_F64 ? gs2dc_applies<double>(sa.A, sa.o) : gs2dc_applies<float>(sa.A, sa.o);
    if (!fits) {
      set_error("the cluster schedule needs a 2-D grid of at least 16 rows whose rows fit 8 CTAs' shared memory, "
                "n_x <= 1024, and no max_blocks");
      return HS_ERR_INVALID;
    }
  }
  // automatic choice: pencils for pipelined batches of one direction when
  // every pencil has a warp of its own (247 against 313 us per sweep at
  // 256^3); single sweeps and symmetric batches are bound by the latency from
  // one pencil to the next and take the large-tile schedule (1.9 against 4.3
  // ms per single sweep), and so do grids with more pencils than resident
  // warps (a warp's second pencil stalls the overlap of sweeps)
  const bool use_pencils = pencils && (sa.o.gs_schedule == 2 || (sa.o.gs_schedule == 0 && !deep));
#define HS_GS(TT, OK)                                                                         \
  if (opk == OK) {                                                                            \
    if (!d3 && (sa.o.gs_schedule == 3 || (sa.o.gs_schedule == 0 && !deep)) &&                  \
        gs2dc_applies<TT>(sa.A, sa.o))                                                        \
      return gs2dc_run_t<TT, OK>(sa, res, hist);                                              \
    if (!d3 && sa.o.gs_schedule != 1 && gs2d_applies<TT>(sa.A, sa.o))                         \
      return gs2d_run_t<TT, OK>(sa, res, hist);                                               \
    if (!d3) return gs_run_t<TT, OK, 2, 0>(sa, res, hist);                                    \
    if constexpr (OK != OP_VARK) {                                                            \
      if (use_pencils && (sa.o.gs_schedule == 2 || gsp_fits<TT, OK>(sa.A, sa.o)))                \
        return gsp_run_t<TT, OK>(sa, res, hist);                                              \
    }                                                                                         \
    return deep ? gs_run_t<TT, OK, 3, 1>(sa, res, hist) : gs_run_t<TT, OK, 3, 0>(sa, res, hist); \
  }
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
