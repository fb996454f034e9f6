// hs_jacobi_tb.cu -- temporally blocked Jacobi: several sweeps per pass over
// the grid (constant-coefficient 7-point operators, 3-D, fixed sweep count).
//
// A pass applies L <= S Jacobi sweeps to one z-chunk of one xy tile while
// reading the input vector once and writing the output once.  Sweep level s
// (level 0 = the input) is kept for three planes in shared memory over the
// tile widened by S - s nodes on every side, so that level s + 1 can be
// formed on a region one node narrower: the widened rings are the
// neighbouring tiles' nodes, recomputed here (the price of not exchanging
// intermediate sweeps through HBM).  Marching up the chunk, plane t of level 0
// is staged, then level s is formed on plane t - s; the z-chunk starts S
// planes early and ends S planes late for the same reason as the rings.
//
// Per node and sweep this trades 24 (FP64) / 12 (FP32) bytes of HBM traffic
// for 24 / L (12 / L) bytes plus the recomputed rings.  On GB300 FP64 Jacobi is
// bound by the FP64 pipe, not by HBM, so blocking pays for FP32 sweeps (memory
// bound) and costs FP64 ones the ring recomputation; both are measured.
//
// Every node runs the same Jacobi-form arithmetic as k_jacobi (jacobi_apply,
// same operand order), so the iterates are bitwise those of single sweeps.
#include <algorithm>
#include <cmath>

#include "hs_krylov.cuh"

namespace hs {

template <typename T>
struct JacTbArgs {
  Geom g;
  Tiling tl;
  Coef<T> cf;      // Jacobi form couplings (g = -a/a_ii)
  T invd;
  const T* b;
  T* bD;           // b / a_ii
  T* x0;           // caller's x
  T* x1;           // ping-pong buffer
  Common cm;
  int sweeps;      // total sweeps
};

// Block layout: one thread per column of the widest region, the tile widened
// by S nodes on every side: (32 + 2S) x (by + 2S) threads (TB_BY = 8 rows).
constexpr int TB_BY = 8;
template <int S>
__host__ __device__ constexpr int tb_w() { return BX + 2 * S; }
template <int S>
__host__ __device__ constexpr int tb_h() { return TB_BY + 2 * S; }
template <int S>
__host__ __device__ constexpr int tb_threads() { return ((tb_w<S>() * tb_h<S>() + 31) / 32) * 32; }
// shared memory: levels 0 .. S-1, two plane buffers each
template <int S>
__host__ __device__ constexpr int tb_smem_values() { return S * 2 * tb_w<S>() * tb_h<S>(); }

// One pass of L sweeps (1 <= L <= S) over one work item, src -> dst.
//
// Thread (tx, ty) owns column (i0 - S + tx, j0 - S + ty) and keeps, per level
// s < S, the column's values at the last three planes in registers (the z
// neighbours); the plane of each level also goes to shared memory, double
// buffered, for the x / y neighbours.  Step t loads level 0 at plane t and
// forms level s at plane t - s inside region s (the tile widened by S - s):
// every shared read of step t is of a plane written in step t - 1, so one
// barrier per step suffices.  The chunk starts S planes early (levels fill
// up) and runs S planes past its end (level S needs level S - 1 one plane up).
template <typename T, int S>
__device__ void tb_item(const JacTbArgs<T>& a, int item, int L, const T* __restrict__ src, T* __restrict__ dst,
                        T* sm) {
  constexpr int W = tb_w<S>(), H = tb_h<S>(), PL = W * H;
  const Geom& g = a.g;
  int i0, j0, z0, z1;
  decode_item(a.tl, g, item, i0, j0, z0, z1);
  const int tx = threadIdx.x % W, ty = threadIdx.x / W;
  const bool live = threadIdx.x < PL;
  const int gi = i0 - S + tx, gj = j0 - S + ty;
  const bool col_in = live && gi >= 0 && gi < g.nx && gj >= 0 && gj < g.ny;
  const long long col = (long long)gj * g.nx + gi;
  const long long P = g.plane;
  const int c = ty * W + tx;
  T q[S][3];   // level s at planes t-s-2, t-s-1, t-s (slots rotate)
#pragma unroll
  for (int s = 0; s < S; s++) q[s][0] = q[s][1] = q[s][2] = T(0);
  // loads run PD planes ahead of their use: the input at plane t + PD, and b/a_ii
  // for planes t - S .. t + PD - 1 (level s at step t needs plane t - s)
  constexpr int PD = 2;
  auto ld_src = [&](int pl) -> T {
    return (col_in && pl >= 0 && pl < g.nz) ? __ldcg(src + (long long)pl * P + col) : T(0);
  };
  auto ld_bd = [&](int pl) -> T {   // bD: written in this kernel, so through L2
    return (col_in && pl >= 0 && pl < g.nz) ? __ldcg(a.bD + (long long)pl * P + col) : T(0);
  };
  const int t0 = z0 - S;
  T srcq[PD], bdq[S + PD];
#pragma unroll
  for (int m = 0; m < PD; m++) srcq[m] = ld_src(t0 + m);
#pragma unroll
  for (int m = 0; m < S + PD; m++) bdq[m] = ld_bd(t0 - S + m);
  for (int t = t0; t <= z1 - 1 + S; t++) {
    // level 0, plane t
    {
      const T v = srcq[0];
#pragma unroll
      for (int m = 0; m + 1 < PD; m++) srcq[m] = srcq[m + 1];
      srcq[PD - 1] = ld_src(t + PD);
      q[0][0] = q[0][1];
      q[0][1] = q[0][2];
      q[0][2] = v;
      if (live) sm[(t & 1) * PL + c] = v;
    }
    // levels 1 .. L on plane t - s, from level s - 1 at planes t - s - 1 .. t - s + 1
#pragma unroll
    for (int s = 1; s <= S; s++) {
      if (s > L) break;
      const int p = t - s;
      const bool in_region = live && tx >= s && tx < W - s && ty >= s && ty < H - s;
      T v = T(0);
      if (in_region && col_in && p >= 0 && p < g.nz) {
        const T* pl = sm + (s - 1) * 2 * PL + (p & 1) * PL;   // level s-1, plane p (written last step)
        Nbr<T> nb;
        nb.c = q[s - 1][1];
        nb.w = pl[c - 1];
        nb.e = pl[c + 1];
        nb.s = pl[c - W];
        nb.n = pl[c + W];
        nb.b = q[s - 1][0];
        nb.t = q[s - 1][2];
        v = jacobi_apply<T, OP_SYM, 3>(a.cf, OpRaw<T, OP_SYM>{}, nb, bdq[S - s]);
        if (s == L && p >= z0 && p < z1 && tx >= S && tx < W - S && ty >= S && ty < H - S)
          dst[(long long)p * P + col] = v;
      }
      if (s < S) {
        q[s][0] = q[s][1];
        q[s][1] = q[s][2];
        q[s][2] = v;
        if (live) sm[s * 2 * PL + (p & 1) * PL + c] = v;
      }
    }
#pragma unroll
    for (int m = 0; m + 1 < S + PD; m++) bdq[m] = bdq[m + 1];
    bdq[S + PD - 1] = ld_bd(t + 1 + PD - 1);
    __syncthreads();
  }
}

template <typename T, int S>
__global__ void __launch_bounds__(tb_threads<S>()) k_jacobi_tb(JacTbArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double sh[32 * MAX_SCAL];
  T* sm = reinterpret_cast<T*>(smraw);
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
    for (long long i = gtid(); i < N; i += gstride()) a.x0[i] = T(0);
    finish(a.cm.ctrl, DS_CONVERGED, 0, 0.0);
    return;
  }
  const T* src = a.x0;
  T* dst = a.x1;
  for (int done = 0; done < a.sweeps;) {
    const int L = min(S, a.sweeps - done);
    for (int item = blockIdx.x; item < a.tl.items(); item += gridDim.x) tb_item<T, S>(a, item, L, src, dst, sm);
    if (!grid_sync(a.cm.ctrl, a.cm.partials, sh)) return;
    done += L;
    T* tmp = const_cast<T*>(src);
    src = dst;
    dst = tmp;
  }
  if (src != a.x0) {
    for (long long i = gtid(); i < N; i += gstride()) a.x0[i] = ldcg(src + i);
  }
  finish(a.cm.ctrl, DS_CONVERGED, a.sweeps, -1.0);
}

template <typename T, int S>
static hs_status jacobi_tb_t(const SolveArgs& sa, hs_result* res, double* hist) {
  const hs_op* A = sa.A;
  const Geom g = geom_of(A);
  Carve c{sa.ws, 0, sa.ws_bytes, true};
  Common cm = carve_common(c, sa.maxit);
  JacTbArgs<T> a = {};
  a.x1 = c.take<T>(g.N);
  a.bD = c.take<T>(g.N);
  if (!c.ok) {
    set_error("workspace too small for Jacobi");
    return HS_ERR_WORKSPACE;
  }
  hs_status s = init_ctrl(cm, sa.o, sa.stream);
  if (s != HS_OK) return s;
  {
    const ConstRow r = const_row(A);
    a.cf.xl = (T)(-r.xl / r.d);
    a.cf.xu = (T)(-r.xu / r.d);
    a.cf.yl = (T)(-r.yl / r.d);
    a.cf.yu = (T)(-r.yu / r.d);
    a.cf.zl = (T)(-r.zl / r.d);
    a.cf.zu = (T)(-r.zu / r.d);
    a.invd = (T)(1.0 / r.d);
  }
  a.g = g;
  a.b = (const T*)sa.b;
  a.x0 = (T*)sa.x;
  a.cm = cm;
  a.sweeps = sa.maxit;
  const int by = TB_BY;
  const int block = tb_threads<S>();
  const size_t smem = (size_t)tb_smem_values<S>() * sizeof(T);
  int per_sm = 0;
  cudaError_t e = cudaFuncSetAttribute(k_jacobi_tb<T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi_tb<T, S>, block, smem);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
  if (per_sm < 1) {
    set_error("temporally blocked Jacobi cannot be resident");
    return HS_ERR_CUDA;
  }
  int grid = std::min(per_sm * sm_count(), MAX_BLOCKS);
  if (sa.o.max_blocks > 0) grid = std::min(grid, sa.o.max_blocks);
  Tiling tl = choose_tiling(g, by, grid, false, sa.o.tile_planes, 1);
  grid = std::max(1, std::min(grid, tl.items()));
  a.tl = tl;
  void* args[] = {&a};
  s = launch_coop((const void*)k_jacobi_tb<T, S>, grid, block, args, smem, sa.stream);
  if (s != HS_OK) return s;
  return finish_solve_pub(sa, cm, nullptr, nullptr, nullptr, nullptr, a.x1, res, hist, false);
}

// Sweeps per pass 2..4 on constant-coefficient 3-D 7-point operators with a
// fixed sweep count (tol = 0); other cases take the one-sweep kernel.
bool jacobi_tb_applies(const SolveArgs& sa) {
  return sa.o.sweeps_per_pass >= 2 && sa.tol == 0.0 && sa.A->ndim == 3 && opkind_of(sa.A) == OP_SYM;
}

hs_status run_jacobi_tb(const SolveArgs& sa, hs_result* res, double* hist) {
  const int S = std::min(sa.o.sweeps_per_pass, 4);
  if (sa.dtype == HS_F64) {
    if (S == 2) return jacobi_tb_t<double, 2>(sa, res, hist);
    if (S == 3) return jacobi_tb_t<double, 3>(sa, res, hist);
    return jacobi_tb_t<double, 4>(sa, res, hist);
  }
  if (S == 2) return jacobi_tb_t<float, 2>(sa, res, hist);
  if (S == 3) return jacobi_tb_t<float, 3>(sa, res, hist);
  return jacobi_tb_t<float, 4>(sa, res, hist);
}

}  // namespace hs
