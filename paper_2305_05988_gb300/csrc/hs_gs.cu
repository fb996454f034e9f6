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
// Two other schedules share the node update (gs_old, then gs_new; hs_gs.cuh):
// the pencil schedule for pipelined batches on 3-D constant-coefficient
// operators (hs_gsp.cu) and, for small 1-/2-D grids, the whole iterate on chip
// in one block or one thread-block cluster (hs_gs2d.cu).  run_gauss_seidel
// below chooses between them.
#include "hs_gs.cuh"

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

// The W = 0 shape has the smaller tiles in every direction.
void gs_counts(const hs_op* A, int* ntiles, int* P) {
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
  if (opkind_of(A) == OP_BOX27) return ((N * es + 255) & ~(size_t)255) + gs27_progress_bytes(A);
  int nt, P;
  gs_counts(A, &nt, &P);
  size_t ints = (size_t)nt + P + 1;
  // b / a_ii, the tile-plane tables, per-tile sweep counts, the claim
  // counter, then the pencil schedule's per-pencil progress counts
  return ((N * es + 255) & ~(size_t)255) + ((ints * 4 + 255) & ~(size_t)255) + (((size_t)nt * 4 + 255) & ~(size_t)255) +
         256 + gsp_progress_bytes(A);
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
    hs_status s = gs_setup<T, OPK>(sa, cm, D, ax, ay, az, a);
    if (s != HS_OK) return s;
  }
  a.plane_off = tabs;
  a.plane_tiles = tabs + P + 1;
  a.ntx = ntx;
  a.nty = nty;
  a.ntz = ntz;
  a.P = P;
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
  return gs_finish<T, OPK>(sa, cm, a, D, ax, ay, az, res, hist);
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
  const bool pencils = gsp_applies(sa);
  if (sa.o.gs_schedule == 2 && !pencils) {
    set_error("the pencil schedule needs a 3-D Laplacian or upwind operator");
    return HS_ERR_INVALID;
  }
  const bool cluster = gs2dc_applies(sa);
  if (sa.o.gs_schedule == 3 && !cluster) {
    set_error("the cluster schedule needs a 2-D grid of at least 16 rows whose rows fit 8 CTAs' shared memory, "
              "n_x <= 1024, and no max_blocks");
    return HS_ERR_INVALID;
  }
  if (!d3) {
    if (cluster && (sa.o.gs_schedule == 3 || (sa.o.gs_schedule == 0 && !deep))) return run_gs2dc(sa, res, hist);
    if (sa.o.gs_schedule != 1 && gs2d_applies(sa)) return run_gs2d(sa, res, hist);
  } else if (pencils && (sa.o.gs_schedule == 2 || (sa.o.gs_schedule == 0 && !deep && gsp_fits(sa)))) {
    // automatic choice: pencils for pipelined batches of one direction when
    // every pencil has a warp of its own (247 against 313 us per sweep at
    // 256^3); single sweeps and symmetric batches are bound by the latency
    // from one pencil to the next and take the large-tile schedule (1.9
    // against 4.3 ms per single sweep), and so do grids with more pencils
    // than resident warps (a warp's second pencil stalls the overlap of
    // sweeps)
    return run_gs_pencils(sa, res, hist);
  }
#define HS_GS(TT, OK)                                                                            \
  if (opk == OK) {                                                                               \
    if (!d3) return gs_run_t<TT, OK, 2, 0>(sa, res, hist);                                       \
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
