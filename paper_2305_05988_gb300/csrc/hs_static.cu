// hs_static.cu -- hs_cg_static: conjugate gradient with library-held scratch.
//
// Some callers cannot allocate device memory: a plug-in running inside a host
// application that hands out all GPU memory through its own pool and does not
// allow foreign cudaMalloc calls, or code on a latency-critical path that must
// not enter an allocator whose cost is unbounded.  hs_cg_static serves them:
// it runs the same CG as hs_cg, but its workspace is a fixed array that lives
// in this library's device image, so the call itself allocates nothing.  The
// caller still provides b and x.
#include <mutex>

#include "hs_internal.h"

// The scratch array.  Every GPU that loads the library holds it until the
// process exits.  In host code `g_static_scratch` is only a stand-in symbol,
// not a device address: its device address is looked up per device below.
static __device__ __align__(256) unsigned char g_static_scratch[HS_STATIC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
// Device address of the scratch array per device, looked up once per process
// on the first call with that device current.  A device reset
// (cudaDeviceReset) while the library is loaded is not supported: the kept
// address would then belong to the destroyed context.
void* g_scratch_dev[kMaxDevices] = {nullptr};
}  // namespace

extern "C" hs_status hs_cg_static(const hs_op* A, hs_dtype dtype, const void* b, void* x, double tol, int maxit,
                                  const hs_opts* opts, void* stream, hs_result* res, double* hist) {
  hs::NvtxRange range("hs_cg_static");
  if (res) {
    res->iters = 0;
    res->status = HS_ERR_INVALID;
    res->rel_res = -1.0;
    res->true_rel_res = -1.0;
    res->restarts = 0;
    res->outer = 0;
    res->inner_iters = 0;
  }
  if (!A) {
    hs::set_error("operator is NULL");
    return HS_ERR_INVALID;
  }
  size_t need = 0;
  hs_status s = hs_workspace_size(A, HS_SOLVER_CG, dtype, opts, maxit, &need);
  if (s != HS_OK) return s;
  if (need > (size_t)HS_STATIC_SCRATCH_BYTES) {
    hs::set_error("hs_cg_static: this problem needs %zu bytes of scratch but the library's static scratch holds "
                  "%zu bytes (HS_STATIC_SCRATCH_BYTES); use hs_cg with a caller workspace",
                  need, (size_t)HS_STATIC_SCRATCH_BYTES);
    return HS_ERR_INVALID;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return hs::cuda_fail(e, "hs_cg_static: cudaGetDevice");
  if (stream) {
    // The scratch address belongs to the current device: a stream of another
    // device would make the solve read memory of the wrong GPU.
    int sdev = -1;
    e = cudaStreamGetDevice((cudaStream_t)stream, &sdev);
    if (e != cudaSuccess) return hs::cuda_fail(e, "hs_cg_static: cudaStreamGetDevice");
    if (sdev != dev) {
      hs::set_error("hs_cg_static: the stream belongs to device %d but device %d is current", sdev, dev);
      return HS_ERR_INVALID;
    }
  }
  if (dev < 0 || dev >= kMaxDevices) {
    hs::set_error("hs_cg_static: device index %d not supported", dev);
    return HS_ERR_INVALID;
  }
  void* ws = nullptr;
  {
    // First call on a device (with that device current): look up the device
    // address of the scratch array once and keep it.
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_dev[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_static_scratch);
      if (e != cudaSuccess) return hs::cuda_fail(e, "hs_cg_static: cudaGetSymbolAddress");
      g_scratch_dev[dev] = p;
    }
    ws = g_scratch_dev[dev];
  }
  // Every section of the workspace that the solver reads before writing (the
  // control block) is initialised by the solver itself at the start of each
  // call, so leftovers from the previous call are harmless.
  return hs_cg(A, dtype, b, x, tol, maxit, opts, ws, (size_t)HS_STATIC_SCRATCH_BYTES, stream, res, hist);
}
