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

template <int S>
__host__ __device__ constexpr int tb_w(int s) { return BX + 2 * (S - s); }
template <int S>
__host__ __device__ inline int tb_h(int by, int s) { return by + 2 * (S - s); }

// Shared-memory values of the level rings (levels 0 .. S-1, 3 planes each).
template <int S>
__host__ __device__ inline int tb_ring_values(int by) {
  int v = 0;
  for (int s = 0; s < S; s++) v += 3 * tb_w<S>(s) * tb_h<S>(by, s);
  return v;
}

template <typename T, int S>
__device__ __forceinline__ T* tb_ring(T* sm, int by, int s) {
  int off = 0;
  for (int q = 0; q < s; q++) off += 3 * tb_w<S>(q) * tb_h<S>(by, q);
  return sm + off;
}

// One pass of L sweeps (1 <= L <= S) over one work item, src -> dst.
template <typename T, int S>
__device__ void tb_item(const JacTbArgs<T>& a, int item, int L, const T* __restrict__ src, T* __restrict__ dst,
                        T* sm) {
  const Geom& g = a.g;
  int i0, j0, z0, z1;
  decode_item(a.tl, g, item, i0, j0, z0, z1);
  const int by = a.tl.by;
  const int nt = blockDim.x;
  const long long P = g.plane;
  for (int t = z0 - L; t <= z1 - 1 + L; t++) {
    // ---- level 0: stage plane t of the input over the widest region
    {
      const int W = tb_w<S>(0), H = tb_h<S>(by, 0);
      T* r0 = tb_ring<T, S>(sm, by, 0) + ((t % 3 + 3) % 3) * W * H;
      const int ib = i0 - S, jb = j0 - S;
      const bool zin = t >= 0 && t < g.nz;
      for (int e = threadIdx.x; e < W * H; e += nt) {
        const int ii = e % W, jj = e / W;
        const int gi = ib + ii, gj = jb + jj;
        T v = T(0);
        if (zin && gi >= 0 && gi < g.nx && gj >= 0 && gj < g.ny) v = __ldcg(src + (long long)t * P + (long long)gj * g.nx + gi);
        r0[e] = v;
      }
    }
    __syncthreads();
    // ---- levels 1 .. L: level s on plane q = t - s from level s-1 planes q-1, q, q+1
    for (int s = 1; s <= L; s++) {
      const int q = t - s;
      const bool out = (s == L);
      // planes of level s this chunk needs: [z0 - (L - s), z1 - 1 + (L - s)]
      const bool need = q >= z0 - (L - s) && q <= z1 - 1 + (L - s);
      if (need) {
        const int lv = s - 1;   // ring of the input level (region widened by S - lv)
        const int Wi = tb_w<S>(lv), Hi = tb_h<S>(by, lv);
        const T* rin = tb_ring<T, S>(sm, by, lv);
        const T* pm = rin + (((q - 1) % 3 + 3) % 3) * Wi * Hi;
        const T* pc = rin + ((q % 3 + 3) % 3) * Wi * Hi;
        const T* pp = rin + (((q + 1) % 3 + 3) % 3) * Wi * Hi;
        // output region: the tile (last level) or the tile widened by S - s
        const int wide = out ? 0 : S - s;
        const int W = BX + 2 * wide, H = by + 2 * wide;
        const int off = (S - lv) - wide;   // input-region coordinates of output (0, 0)
        const bool zin = q >= 0 && q < g.nz;
        T* rout = out ? nullptr : tb_ring<T, S>(sm, by, s) + ((q % 3 + 3) % 3) * W * H;
        for (int e = threadIdx.x; e < W * H; e += nt) {
          const int ii = e % W, jj = e / W;
          const int gi = i0 - wide + ii, gj = j0 - wide + jj;
          const bool in = zin && gi >= 0 && gi < g.nx && gj >= 0 && gj < g.ny;
          T v = T(0);
          if (in) {
            const int c = (jj + off) * Wi + (ii + off);
            Nbr<T> nb;
            nb.c = pc[c];
            nb.w = pc[c - 1];
            nb.e = pc[c + 1];
            nb.s = pc[c - Wi];
            nb.n = pc[c + Wi];
            nb.b = pm[c];
            nb.t = pp[c];
            const long long idx = (long long)q * P + (long long)gj * g.nx + gi;
            v = jacobi_apply<T, OP_SYM, 3>(a.cf, OpRaw<T, OP_SYM>{}, nb, __ldcg(a.bD + idx));   // bD: written in this kernel
            if (out && q >= z0 && q < z1) dst[idx] = v;
          }
          if (!out) rout[e] = v;
        }
      }
      __syncthreads();
    }
  }
}

template <typename T, int S>
__global__ void __launch_bounds__(512) k_jacobi_tb(JacTbArgs<T> a) {
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
  const int by = 8;
  const int block = 32 * by;
  const size_t smem = (size_t)tb_ring_values<S>(by) * sizeof(T);
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
