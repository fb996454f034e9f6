// hs_adjoint.cu -- per-cell gradient of a loss through the diffusion operator.
//
// With A(k) u = f and the adjoint lambda solving A^T lambda = dL/du, the
// derivative of L with respect to the cell coefficient k_i is
//   dL/dk_i = -lambda^T (dA/dk_i) u
//           = -sum_{faces f of cell i} dkappa_f/dk_i (lambda_i - lambda_j)(u_i - u_j) / h_d^2,
// where for an interior face kappa_f = 2 k_i k_j / (k_i + k_j) gives
// dkappa_f/dk_i = 2 k_j^2 / (k_i + k_j)^2, and a boundary face (kappa = k_i,
// lambda_j = u_j = 0) contributes lambda_i u_i / h_d^2.  The kernel writes
// g_i = dL/dlog k_i = k_i dL/dk_i.  (The derivative of L with respect to f is
// lambda itself.)  Not part of the paper: it differentiates the paper's
// diffusion solve for inverse problems.
#include <algorithm>

#include "hs_internal.h"

namespace hs {

template <typename K, int NDIM>
__global__ void __launch_bounds__(256) k_grad_logk(Geom g, const K* __restrict__ kk, const double* __restrict__ u,
                                                   const double* __restrict__ lam, double* __restrict__ out, double ihx,
                                                   double ihy, double ihz) {
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < g.N;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % g.nx);
    const int j = (int)((idx / g.nx) % g.ny);
    const int k = (int)(idx / g.plane);
    const double ki = (double)kk[idx], ui = u[idx], li = lam[idx];
    double acc = 0.0;
    // one face: neighbour at offset off (inside == the face is interior)
    auto face = [&](bool inside, long long off, double ih2) {
      if (inside) {
        const double kj = (double)kk[idx + off];
        const double s = ki + kj;
        const double dk = 2.0 * kj * kj / (s * s);
        acc += dk * (li - lam[idx + off]) * (ui - u[idx + off]) * ih2;
      } else {
        acc += li * ui * ih2;
      }
    };
    face(i > 0, -1, ihx);
    face(i + 1 < g.nx, 1, ihx);
    if (NDIM >= 2) {
      face(j > 0, -(long long)g.nx, ihy);
      face(j + 1 < g.ny, (long long)g.nx, ihy);
    }
    if (NDIM >= 3) {
      face(k > 0, -g.plane, ihz);
      face(k + 1 < g.nz, g.plane, ihz);
    }
    out[idx] = -ki * acc;
  }
}

template <typename K>
static hs_status launch_grad(const hs_op* A, const double* u, const double* lam, double* gout, cudaStream_t st) {
  Geom g = geom_of(A);
  double ih[3];
  for (int d = 0; d < 3; d++) ih[d] = d < A->ndim ? 1.0 / (A->h[d] * A->h[d]) : 0.0;
  int blocks = (int)std::max<long long>(1, std::min<long long>((g.N + 255) / 256, (long long)sm_count() * 16));
  const K* kk = (const K*)A->k;
  if (A->ndim >= 3)
    k_grad_logk<K, 3><<<blocks, 256, 0, st>>>(g, kk, u, lam, gout, ih[0], ih[1], ih[2]);
  else if (A->ndim == 2)
    k_grad_logk<K, 2><<<blocks, 256, 0, st>>>(g, kk, u, lam, gout, ih[0], ih[1], ih[2]);
  else
    k_grad_logk<K, 1><<<blocks, 256, 0, st>>>(g, kk, u, lam, gout, ih[0], ih[1], ih[2]);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HS_OK : cuda_fail(e, "gradient launch");
}

// k_i = exp(log k_i): the diffusion coefficient from its logarithm, the
// parametrisation in which the gradient above is taken.
__global__ void __launch_bounds__(256) k_exp_logk(const double* logk, double* k, long long n) {
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x)
    k[idx] = exp(logk[idx]);
}

}  // namespace hs

extern "C" hs_status hs_exp_logk(const double* logk, double* k, int64_t n, void* stream) {
  if (n < 0 || (n > 0 && (!logk || !k))) {
    hs::set_error("hs_exp_logk: NULL vector or negative length");
    return HS_ERR_INVALID;
  }
  if (n == 0) return HS_OK;
  if (k != logk && ((k < logk && k + n > logk) || (logk < k && logk + n > k))) {
    hs::set_error("hs_exp_logk: k overlaps logk without being the same array");
    return HS_ERR_INVALID;
  }
  int blocks = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, (long long)hs::sm_count() * 16));
  hs::k_exp_logk<<<blocks, 256, 0, (cudaStream_t)stream>>>(logk, k, (long long)n);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HS_OK : hs::cuda_fail(e, "exp(log k) launch");
}

extern "C" hs_status hs_diffusion_grad_logk(const hs_op* A, const double* u, const double* lam, double* g,
                                            void* stream) {
  hs::NvtxRange range("hs_diffusion_grad_logk");
  if (!A || !u || !lam || !g) {
    hs::set_error("NULL argument");
    return HS_ERR_INVALID;
  }
  if (A->kind != hs::KIND_DIFFUSION) {
    hs::set_error("hs_diffusion_grad_logk needs a diffusion operator");
    return HS_ERR_INVALID;
  }
  if (g == u || g == lam) {
    hs::set_error("g must not alias u or lam");
    return HS_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (A->kdt == HS_F64) return hs::launch_grad<double>(A, u, lam, g, st);
  return hs::launch_grad<float>(A, u, lam, g, st);
}
