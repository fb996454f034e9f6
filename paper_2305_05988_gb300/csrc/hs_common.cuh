// hs_common.cuh -- device-side building blocks shared by the libhsolve kernels:
// the stencil descriptor, deterministic block reductions, and the bounded
// grid "reduce-barrier" used by the persistent solver kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hs {

// ---------------------------------------------------------------------------
// Debug builds (-DHS_DEBUG): every global index the tile engines compute is
// checked against the vector length before it is used; a bad index is
// recorded (1 + index, first one wins) in a word of this translation unit and
// the access is skipped -- no trap, no assert, the kernel runs on.  The host
// launchers read and clear the word after each solve (hs_dbg_take) and return
// HS_ERR_BOUNDS.  In release builds HS_IN_BOUNDS is constant true.
// ---------------------------------------------------------------------------
#ifdef HS_DEBUG
static __device__ unsigned long long hs_dbg_word;
__device__ __forceinline__ bool hs_in_bounds(long long idx, long long n) {
  if (idx >= 0 && idx < n) return true;
  atomicCAS(&hs_dbg_word, 0ull, 1ull + (unsigned long long)idx);
  return false;
}
#define HS_IN_BOUNDS(idx, n) hs_in_bounds((long long)(idx), (long long)(n))
#else
#define HS_IN_BOUNDS(idx, n) true
#endif

// Operator kinds as compiled into kernels.
// OP_BOX27: the HPCG 27-point system (diagonal 27, -1 on the 26 neighbours of
// the 3x3x3 box), applied through separable box sums (3-D only).
enum OpKind : int { OP_SYM = 0, OP_NONSYM = 1, OP_VARK = 2, OP_BOX27 = 3 };

// Device status word values (mirrors hs_status where they overlap).
enum DevStatus : int {
  DS_RUNNING = 0,
  DS_CONVERGED = 1,
  DS_MAXIT = 2,
  DS_BREAKDOWN = -3,
  DS_NONFINITE = -4,
  DS_TIMEOUT = -5,
};

// Stencil coefficients.  A row reads
//   y_i = d c + xl W + xu E + yl S + yu N + zl B + zu T
// (W/E = i -+ 1, S/N = j -+ 1, B/T = k -+ 1, out-of-grid values are zero).
// OP_SYM keeps xl == xu etc. so that pairs can be summed first.  OP_VARK
// reads per-cell coefficients: D[i] on the diagonal and the lower-face
// couplings ax/ay/az (positive), the upper faces taken from the neighbour's
// lower face:  y_i = D_i c - ax_i W - ax_{i+1} E - ay_i S - ay_{i+nx} N
//                         - az_i B - az_{i+nx ny} T.
template <typename T>
struct Coef {
  T d, xl, xu, yl, yu, zl, zu;
  const T* D;
  const T* ax;
  const T* ay;
  const T* az;
};

struct Geom {
  int nx, ny, nz;      // nz = 1 for 2-D, ny = nz = 1 for 1-D
  long long N;
  long long plane;     // nx * ny
};

// ---------------------------------------------------------------------------
// Exact binary32 -> binary64 widening with integer operations.  On this GPU
// the F2F.F64.F32 conversion instruction issues on the FP64 pipe (measured at
// about the FP64 FMA rate), so the FP64-accumulated dot products of FP32
// vectors build the binary64 bit pattern from the binary32 fields instead:
// exponent rebiased by 1023 - 127 = 896, fraction shifted left by 29.  Normal
// numbers, zeros, infinities and NaNs are widened exactly; binary32
// subnormals (magnitude below 2^-126) are flushed to zero.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double widen(double d) { return d; }
__device__ __forceinline__ double widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ef = (u >> 23) & 0xffu;
  const unsigned de = (ef == 0u) ? 0u : (ef == 255u ? 2047u : ef + 896u);
  const unsigned m = (ef == 0u) ? 0u : (u & 0x7fffffu);
  const unsigned hi = (u & 0x80000000u) | (de << 20) | (m >> 3);
  const unsigned lo = (m & 7u) << 29;
  return __hiloint2double((int)hi, (int)lo);
}

// ---------------------------------------------------------------------------
// Deterministic reductions.  Every sum below is taken in a fixed order that
// depends only on the launch shape, never on timing, so repeated solves give
// bit-identical scalars.
// ---------------------------------------------------------------------------

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sums of NS values; result valid in every thread.  `sh` must hold
// at least 32 * NS doubles.  Contains __syncthreads(): call from all threads.
template <int NS>
__device__ __forceinline__ void block_sum(double (&v)[NS], double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarp = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int s = 0; s < NS; s++) v[s] = warp_sum(v[s]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int s = 0; s < NS; s++) sh[s * 32 + warp] = v[s];
  }
  __syncthreads();
#pragma unroll
  for (int s = 0; s < NS; s++) {
    double t = (lane < nwarp) ? sh[s * 32 + lane] : 0.0;
    v[s] = warp_sum(t);
  }
  __syncthreads();
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed(unsigned* p, unsigned v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire_int(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Control block at the start of every solver workspace (zeroed by the host
// before each solve).
struct Ctrl {
  unsigned count;        // blocks arrived at the current barrier
  unsigned gen;          // barrier generation
  int status;            // DevStatus
  int iters;             // iterations completed
  int restarts;          // BiCGStab restarts
  int pad0;
  unsigned long long timeout_ns;
  double scal[16];       // reduced scalars of the last barrier
  double rel_res;        // last relative residual
  double aux[7];
};

static_assert(sizeof(Ctrl) <= 512, "Ctrl must fit its 512-byte slot");

// A team is the set of blocks that solve one system together: rank and size
// within the team, and the team's own control block and partial-sum slots.
// A standalone solve uses the whole grid as one team; the batched solver runs
// many teams (one per large system, single-block teams for small ones) in
// one cooperative launch.
struct Team {
  int rank;
  int size;
  Ctrl* ctrl;
  double* partials;   // size * NS doubles
  __device__ __forceinline__ long long tid() const { return (long long)rank * blockDim.x + threadIdx.x; }
  __device__ __forceinline__ long long stride() const { return (long long)size * blockDim.x; }
  __device__ __forceinline__ bool lead() const { return rank == 0 && threadIdx.x == 0; }
};

__device__ __forceinline__ Team grid_team(Ctrl* ctrl, double* partials) {
  Team t;
  t.rank = blockIdx.x;
  t.size = gridDim.x;
  t.ctrl = ctrl;
  t.partials = partials;
  return t;
}

// Team reduce-barrier.  Every block of the team contributes NS partial sums
// (already block-reduced, valid in thread 0), the last block to arrive sums
// all partials in rank order (so the result does not depend on arrival order),
// publishes them in ctrl->scal and releases the others.  All threads of all
// team blocks return the same NS doubles in `out`.  Returns false if the wait
// ran out (ctrl->status is then DS_TIMEOUT) or another block flagged an error;
// the caller must then stop working on this team's solve.
//
// All blocks of the team must be co-resident (cooperative launch).  `sh` needs
// 32 * NS doubles of shared memory.
template <int NS>
__device__ bool team_reduce(const Team& tm, const double (&mine)[NS], double (&out)[NS], double* sh) {
  __shared__ int s_last;
  __shared__ int s_ok;
  Ctrl* ctrl = tm.ctrl;
  double* partials = tm.partials;
  const int tid = threadIdx.x;
  if (tid == 0) {
    unsigned g = ld_acquire(&ctrl->gen);
#pragma unroll
    for (int s = 0; s < NS; s++) partials[(size_t)tm.rank * NS + s] = mine[s];
    __threadfence();
    unsigned arrived = atomicAdd(&ctrl->count, 1u);
    s_last = (arrived == (unsigned)tm.size - 1);
    s_ok = 1;
    if (!s_last) {
      unsigned long long t0 = global_ns();
      unsigned spins = 0;
      while (ld_acquire(&ctrl->gen) == g) {
        if (++spins > 64) {
          __nanosleep(100);
          if ((spins & 255) == 0) {
            if (ld_acquire_int(&ctrl->status) < 0) { s_ok = 0; break; }
            if (global_ns() - t0 > ctrl->timeout_ns) {
              atomicCAS(&ctrl->status, 0, (int)DS_TIMEOUT);
              s_ok = 0;
              break;
            }
          }
        }
      }
    }
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    double acc[NS];
#pragma unroll
    for (int s = 0; s < NS; s++) acc[s] = 0.0;
    for (int b = tid; b < tm.size; b += blockDim.x) {
#pragma unroll
      for (int s = 0; s < NS; s++) acc[s] += __ldcg(&partials[(size_t)b * NS + s]);
    }
    block_sum<NS>(acc, sh);
    if (tid == 0) {
#pragma unroll
      for (int s = 0; s < NS; s++) ctrl->scal[s] = acc[s];
      ctrl->count = 0;
      __threadfence();
      unsigned g = ctrl->gen;
      st_release(&ctrl->gen, g + 1);
    }
#pragma unroll
    for (int s = 0; s < NS; s++) out[s] = acc[s];
    __syncthreads();
    return ld_acquire_int(&ctrl->status) >= 0;
  }
  int ok = s_ok;
  __syncthreads();
  if (!ok) return false;
#pragma unroll
  for (int s = 0; s < NS; s++) out[s] = __ldcg(&ctrl->scal[s]);
  __syncthreads();
  return true;
}

// Whole-grid forms used by the standalone solver kernels.
template <int NS>
__device__ __forceinline__ bool grid_reduce(Ctrl* ctrl, double* partials, const double (&mine)[NS],
                                            double (&out)[NS], double* sh) {
  return team_reduce<NS>(grid_team(ctrl, partials), mine, out, sh);
}

// Plain barriers (no data).
__device__ __forceinline__ bool team_sync(const Team& tm, double* sh) {
  double z[1] = {0.0}, o[1];
  return team_reduce<1>(tm, z, o, sh);
}
__device__ __forceinline__ bool grid_sync(Ctrl* ctrl, double* partials, double* sh) {
  return team_sync(grid_team(ctrl, partials), sh);
}

}  // namespace hs
