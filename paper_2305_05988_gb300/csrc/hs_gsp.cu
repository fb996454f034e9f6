// hs_gsp.cu -- the pencil schedule of exactly lexicographic Gauss-Seidel
// (section 3.1) on 3-D constant-coefficient operators.  A warp owns a pencil of
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
// the tile schedule (gs_old then gs_new, hs_gs.cuh), so iterates are bitwise those of the tile
// schedule.
#include "hs_gs.cuh"

namespace hs {

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
// Host side
// ---------------------------------------------------------------------------

// The pencil schedule applies to 3-D constant-coefficient operators whose
// progress counts (sweeps x pairs per line) fit in 32 bits.
bool gsp_applies(const SolveArgs& sa) {
  const hs_op* A = sa.A;
  if (A->ndim != 3) return false;
  const int opk = opkind_of(A);
  if (opk != OP_SYM && opk != OP_NONSYM) return false;
  const long long nq = (A->n[0] + 1) / 2;
  const long long sweeps = (long long)sa.maxit * (sa.o.gs_mode == HS_GS_SYMMETRIC ? 2 : 1) + 2;
  return sweeps * nq < (1ll << 31);
}

// Whether every pencil gets a warp of its own (so that sweeps overlap), and
// there are enough of them to keep at least twelve warps busy on every SM (with
// fewer, the FP64 pipe idles behind each warp's dependent chain: 192^3 runs
// 153 us per sweep against 142 with tiles).
template <typename T, int OPK>
static bool gsp_fits_t(const hs_op* A, const hs_opts& o) {
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
    hs_status s = gs_setup<T, OPK>(sa, cm, nullptr, nullptr, nullptr, nullptr, a);
    if (s != HS_OK) return s;
  }
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
  return gs_finish<T, OPK>(sa, cm, a, nullptr, nullptr, nullptr, nullptr, res, hist);
}

bool gsp_fits(const SolveArgs& sa) {
  const bool sym = opkind_of(sa.A) == OP_SYM;
  if (sa.dtype == HS_F64) return sym ? gsp_fits_t<double, OP_SYM>(sa.A, sa.o) : gsp_fits_t<double, OP_NONSYM>(sa.A, sa.o);
  return sym ? gsp_fits_t<float, OP_SYM>(sa.A, sa.o) : gsp_fits_t<float, OP_NONSYM>(sa.A, sa.o);
}

// Per-pencil progress counts and the zero words read in place of values
// outside the grid.
size_t gsp_progress_bytes(const hs_op* A) {
  const size_t npen = (size_t)((A->n[1] + GSP_PY - 1) / GSP_PY) * (size_t)((A->n[2] + GSP_PZ - 1) / GSP_PZ);
  return ((npen * 4 + 255) & ~(size_t)255) + 256;
}

hs_status run_gs_pencils(const SolveArgs& sa, hs_result* res, double* hist) {
  if (!gsp_applies(sa)) {
    set_error("the pencil schedule needs a 3-D Laplacian or upwind operator");
    return HS_ERR_INVALID;
  }
  const bool sym = opkind_of(sa.A) == OP_SYM;
  if (sa.dtype == HS_F64) return sym ? gsp_run_t<double, OP_SYM>(sa, res, hist) : gsp_run_t<double, OP_NONSYM>(sa, res, hist);
  return sym ? gsp_run_t<float, OP_SYM>(sa, res, hist) : gsp_run_t<float, OP_NONSYM>(sa, res, hist);
}

}  // namespace hs
