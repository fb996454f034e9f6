// hs_batch_mixed.cu -- mixed-precision variant of the batched persistent
// solver: every system runs FP64 iterative refinement with an FP32 inner
// Krylov solve, the whole refinement of a system inside one job of the
// cooperative kernel (teams and queue as in hs_batch.cu).
//
// Refinement step of one system (team of blocks, all decisions taken from
// the same reduced scalars):
//   r = b - A x in FP64 (FP64 operator), written as r32 = fl32(s r) with a
//   power-of-two scale s (exact) that keeps FP32 entries near unit size;
//   ||r||, ||b|| reduced in FP64; stop when ||r|| / ||b|| <= tol;
//   solve A d = r32 in FP32 from d = 0 to the inner tolerance (FP32 vectors
//   and coefficients, FP64-accumulated dots): the standalone CG / BiCGStab
//   iteration bodies, run by the same team on the system's inner control block;
//   x += d / s in FP64, d = 0.
#include <algorithm>
#include <cmath>

#include "hs_batch.cuh"

namespace hs {

// r = b - sigma A x (FP64), stored scaled and rounded to FP32.
template <int OPK, int NDIM>
struct ResF32Sink {
  Coef<double> cf;
  Geom g;
  double sigma;
  const double* b;
  float* r32;
  double scale;
  double acc[2];
  struct Raw {
    OpRaw<double, OPK> o;
    double b;
  };
  __device__ __forceinline__ Raw fetch(long long idx, int i, int j, int k) const {
    return Raw{op_fetch<double, OPK, NDIM>(cf, g, idx, i, j, k), __ldg(b + idx)};
  }
  __device__ __forceinline__ void operator()(long long idx, const Nbr<double>& nb, const Raw& q, int, int, int) {
    const double v = op_apply<double, OPK, NDIM>(cf, q.o, nb);
    const double rv = (OPK == OP_VARK) ? q.b - v : fma(-sigma, v, q.b);
    r32[idx] = (float)(rv * scale);
    acc[0] += rv * rv;
    acc[1] += q.b * q.b;
  }
};

// 2^-e with 2^e nearest below |v| (v > 0 and finite); 1 otherwise.
__device__ __forceinline__ double pow2_inverse(double v) {
  if (!(v > 0.0) || !isfinite(v)) return 1.0;
  return ldexp(1.0, -ilogb(v));
}

template <int OPK, int NDIM, bool BI>
__device__ void mx_body(MxSys& a, const Team& tm, unsigned char* smraw, double* sh) {
  double* sm64 = reinterpret_cast<double*>(smraw);
  float* sm32 = reinterpret_cast<float*>(smraw);
  const long long N = a.g.N;
  Team ti = tm;
  ti.ctrl = a.inner_ctrl;

  // d = 0 and the scale of the first residual (from the RMS of b)
  double bb0[1];
  {
    double acc[1] = {0.0};
    for (long long i = tm.tid(); i < N; i += tm.stride()) {
      const double bv = __ldg(a.b + i);
      acc[0] += bv * bv;
      a.d32[i] = 0.0f;
    }
    block_sum<1>(acc, sh);
    if (!team_reduce<1>(tm, acc, bb0, sh)) return;
  }
  double scale = pow2_inverse(sqrt(bb0[0] / (double)N));
  double bb = 0.0, rel = -1.0;
  long long inner_total = 0;
  int outer = 0, status = DS_MAXIT, restarts = 0;
  for (;; outer++) {
    ResF32Sink<OPK, NDIM> sink{a.cf, a.g, a.sigma, a.b, a.r32, scale, {0.0, 0.0}};
    LoadSrc<double, true> src{a.x};
    for (int item = tm.rank; item < a.tl.items(); item += tm.size)
      zmarch_item<double, NDIM, BATCH_CX>(a.g, a.tl, item, sm64, src, sink);
    block_sum<2>(sink.acc, sh);
    double s2[2];
    if (!team_reduce<2>(tm, sink.acc, s2, sh)) return;
    if (outer == 0) bb = s2[1];
    if (bb == 0.0) {
      for (long long i = tm.tid(); i < N; i += tm.stride()) a.x[i] = 0.0;
      rel = 0.0;
      status = DS_CONVERGED;
      break;
    }
    rel = sqrt(s2[0] / bb);
    if (!isfinite(rel)) {
      status = DS_NONFINITE;
      break;
    }
    if (rel <= a.tol) {
      status = DS_CONVERGED;
      break;
    }
    if (outer >= a.max_outer) break;
    // inner FP32 solve of A d = r32; BiCGStab's absolute restart threshold
    // is applied to the unit-norm right-hand side, as in the standalone
    // mixed solver: scale it by ||r32||
    // a step close to tol stops its inner solve once tol is within reach
    // (the same decision in every block of the team: rel is team-reduced)
    {
      const double itol = a.inner_fixed ? a.inner_tol : inner_tol_for(a.inner_tol, a.tol, rel);
      if (threadIdx.x == 0) {
        if constexpr (BI) {
          a.bi.reps = a.restart_eps * sqrt(s2[0]) * scale;
          a.bi.tol = itol;
        } else {
          a.cg.tol = itol;
        }
      }
      __syncthreads();
    }
    BodyOut io;
    if constexpr (BI)
      io = bicgstab_body<float, OPK, NDIM, BATCH_CX>(a.bi, ti, sm32, sh);
    else
      io = cg_body<float, OPK, NDIM, BATCH_CX>(a.cg, ti, sm32, sh);
    if (!io.ok) {
      if (tm.lead()) atomicCAS(&tm.ctrl->status, 0, (int)DS_TIMEOUT);
      return;
    }
    inner_total += io.iters;
    restarts += io.restarts;
    if (io.status == DS_NONFINITE) {
      status = DS_NONFINITE;
      break;
    }
    // x += d / s ; d = 0  (a breakdown or an unconverged inner solve still
    // gives a usable correction: the next FP64 residual decides)
    const double inv = 1.0 / scale;
    for (long long i = tm.tid(); i < N; i += tm.stride()) {
      a.x[i] = fma((double)a.d32[i], inv, a.x[i]);
      a.d32[i] = 0.0f;
    }
    if (!team_sync(tm, sh)) return;
    scale = pow2_inverse(sqrt(s2[0] / (double)N));
  }
  if (tm.lead()) {
    tm.ctrl->aux[0] = (double)inner_total;
    tm.ctrl->aux[1] = (double)outer;
    tm.ctrl->restarts = restarts;
  }
  team_finish(tm, status, outer, rel);
}

__device__ __forceinline__ void mx_job(const MxSys* __restrict__ sys, int s, int rank, int size, MxSys& d,
                                       unsigned char* smraw, double* sh) {
  {
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(sys + s);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(&d);
    for (int w = threadIdx.x; w < (int)(sizeof(MxSys) / 8); w += blockDim.x) dst[w] = src[w];
  }
  __syncthreads();
  Team tm;
  tm.rank = rank;
  tm.size = size;
  tm.ctrl = d.cm.ctrl;
  tm.partials = d.cm.partials;
  switch (d.kind) {
    case MK_CG_SYM2: mx_body<OP_SYM, 2, false>(d, tm, smraw, sh); break;
    case MK_CG_SYM3: mx_body<OP_SYM, 3, false>(d, tm, smraw, sh); break;
    case MK_CG_VARK2: mx_body<OP_VARK, 2, false>(d, tm, smraw, sh); break;
    case MK_CG_VARK3: mx_body<OP_VARK, 3, false>(d, tm, smraw, sh); break;
    case MK_BI_SYM2: mx_body<OP_SYM, 2, true>(d, tm, smraw, sh); break;
    case MK_BI_SYM3: mx_body<OP_SYM, 3, true>(d, tm, smraw, sh); break;
    case MK_BI_NONSYM2: mx_body<OP_NONSYM, 2, true>(d, tm, smraw, sh); break;
    case MK_BI_NONSYM3: mx_body<OP_NONSYM, 3, true>(d, tm, smraw, sh); break;
    case MK_BI_VARK2: mx_body<OP_VARK, 2, true>(d, tm, smraw, sh); break;
    default: mx_body<OP_VARK, 3, true>(d, tm, smraw, sh); break;
  }
  __syncthreads();
}

// Team jobs first, then single-block systems from the largest-first queue
// (the scheme of the FP64 batch kernel).
__global__ void __launch_bounds__(BATCH_THREADS, HS_BATCHMX_MINBLOCKS) k_batch_mx(const MxSys* __restrict__ sys,
                                                            const int* __restrict__ job_off,
                                                            const BatchJob* __restrict__ jobs,
                                                            const int* __restrict__ queue, int nqueue,
                                                            int* __restrict__ head) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double sh[32 * MAX_SCAL];
  __shared__ MxSys d;
  __shared__ int s_next;
  for (int j = job_off[blockIdx.x]; j < job_off[blockIdx.x + 1]; j++) {
    const BatchJob jb = jobs[j];
    mx_job(sys, jb.sys, jb.rank, jb.size, d, smraw, sh);
  }
  for (;;) {
    if (threadIdx.x == 0) s_next = atomicAdd(head, 1);
    __syncthreads();
    const int q = s_next;
    __syncthreads();
    if (q >= nqueue) break;
    mx_job(sys, queue[q], 0, 1, d, smraw, sh);
  }
}

__device__ __forceinline__ void ctrl_reset(Ctrl* c, unsigned long long timeout_ns) {
  c->count = 0;
  c->gen = 0;
  c->status = 0;
  c->iters = 0;
  c->restarts = 0;
  c->timeout_ns = timeout_ns;
  c->rel_res = -1.0;
  c->aux[0] = 0.0;
  c->aux[1] = 0.0;
}

__global__ void k_batch_mx_init(const MxSys* __restrict__ sys, int nsys, unsigned long long timeout_ns, int* head) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *head = 0;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsys; s += gridDim.x * blockDim.x) {
    ctrl_reset(sys[s].cm.ctrl, timeout_ns);
    ctrl_reset(sys[s].inner_ctrl, timeout_ns);
  }
}

__global__ void k_batch_mx_gather(const MxSys* __restrict__ sys, int nsys, double* __restrict__ out) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsys; s += gridDim.x * blockDim.x) {
    const Ctrl* c = sys[s].cm.ctrl;
    double* o = out + (size_t)BATCH_OUT * s;
    o[0] = (double)c->status;
    o[1] = (double)c->iters;
    o[2] = c->rel_res;
    o[3] = (double)c->restarts;
    o[4] = c->aux[1];
    o[5] = c->aux[0];
  }
}

int batch_mx_blocks_per_sm(int threads, size_t smem) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_mx, threads, smem) != cudaSuccess) return 0;
  return per_sm;
}

cudaError_t batch_mx_launch(cudaStream_t s, int grid, size_t smem, const MxSys* sys, int nsys,
                            unsigned long long timeout_ns, const int* job_off, const BatchJob* jobs, const int* queue,
                            int nqueue, int* head, double* out) {
  const int ib = std::max(1, std::min(64, (nsys + 255) / 256));
  k_batch_mx_init<<<ib, 256, 0, s>>>(sys, nsys, timeout_ns, head);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(BATCH_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_batch_mx, sys, job_off, jobs, queue, nqueue, head);
  if (e != cudaSuccess) return e;
  k_batch_mx_gather<<<ib, 256, 0, s>>>(sys, nsys, out);
  return cudaGetLastError();
}

}  // namespace hs
