// hs_diag.cu -- hs_diag_fp64_rate: the FP64 fused multiply-add rate this GPU
// sustains, measured with independent dependency chains in every thread.  The
// FP64 solvers of this library are bound by that rate (a 7-point FP64 stencil
// needs about 6 FP64 instructions per node, more than its 24 bytes of traffic
// allow at HBM speed on this part), so the benchmark divides their flop rates
// by this measurement.
#include "hs_internal.h"

namespace hs {

namespace {

constexpr int kChains = 8;       // independent FMA chains per thread
constexpr int kBlock = 256;

// Each thread runs kChains dependent DFMA chains of `iters` steps; the
// chains are independent of each other so the FP64 pipe can interleave them.
// The result is stored so the work is not removed.
__global__ void __launch_bounds__(kBlock) k_fp64_rate(double* out, int iters, double a, double b) {
  double v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; c++) v[c] = (double)(threadIdx.x + c) * 1e-3;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int c = 0; c < kChains; c++) v[c] = fma(v[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; c++) s += v[c];
  if (s == 12345.678) out[0] = s;   // practically never true: keeps the chains live
  if (threadIdx.x == 0 && blockIdx.x == 0) out[1] = s;
}

}  // namespace

}  // namespace hs

using namespace hs;

extern "C" hs_status hs_diag_fp64_rate(void* stream, double* flops_per_s) {
  if (!flops_per_s) {
    set_error("flops_per_s is NULL");
    return HS_ERR_INVALID;
  }
  *flops_per_s = 0.0;
  cudaStream_t st = (cudaStream_t)stream;
  double* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, 2 * sizeof(double));
  if (e != cudaSuccess) return cuda_fail(e, "diagnostic buffer");
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_rate, kBlock, 0);
  const int grid = sm_count() * (per_sm > 0 ? per_sm : 1);
  const int iters = 4096;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  hs_status s = HS_OK;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best_ms = 1e30f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; rep++) {   // the first launch warms up
    e = cudaEventRecord(e0, st);
    if (e != cudaSuccess) break;
    k_fp64_rate<<<grid, kBlock, 0, st>>>(buf, iters, 0.999999, 1e-9);
    e = cudaGetLastError();
    if (e != cudaSuccess) break;
    e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && ms < best_ms) best_ms = ms;
  }
  if (e != cudaSuccess) s = cuda_fail(e, "FP64 rate kernel");
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaError_t ef = cudaFree(buf);
  if (s != HS_OK) return s;
  if (ef != cudaSuccess) return cuda_fail(ef, "diagnostic buffer");
  // 2 flops per FMA
  *flops_per_s = 2.0 * (double)grid * kBlock * kChains * (double)iters / (best_ms * 1e-3);
  return HS_OK;
}
