// hs_internal.h -- host-side internals shared by the libhsolve translation
// units (operator descriptor, solve context, workspace carving, launchers).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include <string>

#include "../../include/hsolve.h"
#include "hs_common.cuh"
#include "hs_stencil.cuh"

struct hs_grid {
  int ndim;
  int64_t n[3];
};

struct hs_op {
  int ndim;
  int kind;           // 0 Laplacian, 1 upwind, 2 diffusion
  int64_t n[3];       // unused dimensions = 1
  double h[3];
  double beta[3];
  const void* k;      // diffusion: borrowed device pointer
  int kdt;            // hs_dtype of k
};

namespace hs {

// KIND_HPCG7 / KIND_HPCG27: the paper's benchmark system (section 4.1),
// diagonal 27 and -1 for each face (7) or box (27) neighbour, unscaled.
enum { KIND_LAPLACIAN = 0, KIND_UPWIND = 1, KIND_DIFFUSION = 2, KIND_HPCG7 = 3, KIND_HPCG27 = 4 };

// An NVTX range around each public call (header-only NVTX 3: a no-op unless
// a profiler is attached), so that profiles and ncu's --nvtx filters can pick
// out one solve: "hs_cg", "hs_bicgstab", ...
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

void set_error(const char* fmt, ...);
hs_status cuda_fail(cudaError_t e, const char* what);

// Debug builds: the bounds-check word of the calling translation unit
// (hs_common.cuh), read and cleared after `st` has drained; HS_ERR_BOUNDS if
// a check fired.  Release builds: HS_OK.
static inline hs_status hs_dbg_take(cudaStream_t st) {
#ifdef HS_DEBUG
  unsigned long long w = 0;
  cudaError_t e = cudaMemcpyFromSymbolAsync(&w, hs_dbg_word, sizeof(w), 0, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "debug word read-back");
  if (w) {
    const unsigned long long zero = 0;
    cudaMemcpyToSymbolAsync(hs_dbg_word, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, st);
    cudaStreamSynchronize(st);
    set_error("debug bounds check: global index %lld out of range", (long long)(w - 1));
    return HS_ERR_BOUNDS;
  }
#else
  (void)st;
#endif
  return HS_OK;
}

inline int opkind_of(const hs_op* A) {
  if (A->kind == KIND_DIFFUSION) return OP_VARK;
  if (A->kind == KIND_HPCG27) return OP_BOX27;
  if (A->kind == KIND_UPWIND) {
    for (int d = 0; d < A->ndim; d++)
      if (A->beta[d] != 0.0) return OP_NONSYM;
  }
  return OP_SYM;
}

inline Geom geom_of(const hs_op* A) {
  Geom g;
  g.nx = (int)A->n[0];
  g.ny = (int)A->n[1];
  g.nz = (int)A->n[2];
  g.plane = (long long)g.nx * g.ny;
  g.N = g.plane * g.nz;
  return g;
}

// Unscaled constant row of an operator: diagonal and the six couplings
// (lower/upper per dimension; missing dimensions give zeros).
struct ConstRow {
  double d, xl, xu, yl, yu, zl, zu;
};
ConstRow const_row(const hs_op* A);

// Chooses a tiling (rows per tile, z chunk length) for `grid` persistent
// blocks, or for a one-item-per-block launch when grid == 0.
Tiling choose_tiling(const Geom& g, int by, int grid, bool src_expensive, int planes = 0, int cx = 1);

// Workspace carving: every section is 256-byte aligned.
struct Carve {
  char* base;
  size_t off;
  size_t cap;
  bool ok;
  template <typename T>
  T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~(size_t)255;
    if (off + bytes > cap) ok = false;
    T* p = base ? (T*)(base + off) : nullptr;
    off += bytes;
    return p;
  }
};

constexpr int MAX_BLOCKS = 4096;   // cap on persistent grid size
constexpr int MAX_SCAL = 4;        // scalars per grid reduction

struct Common {
  Ctrl* ctrl;
  double* partials;
  double* hist;      // device, maxit + 2 entries
};

size_t common_bytes(int maxit);
Common carve_common(Carve& c, int maxit);

struct SolveArgs {
  const hs_op* A;
  hs_dtype dtype;
  const void* b;
  void* x;
  double tol;
  int maxit;
  hs_opts o;
  char* ws;
  size_t ws_bytes;
  cudaStream_t stream;
  // asynchronous form (hs_*_async): the result and the history are written
  // by a kernel into device memory and nothing on the host waits
  bool async_dev = false;
  hs_result* res_dev = nullptr;
  double* hist_dev = nullptr;
};

// Doubles of the BiCGStab restart trace section (r_k . r' and a restart flag
// for k = 0 .. maxit, plus one spare pair).
inline size_t bicgstab_trace_len(int maxit) { return 2 * ((size_t)maxit + 2); }

// Inner relative tolerance of one mixed-precision refinement step whose FP64
// relative residual is rel: the step has to bring the residual from rel to
// tol, so its inner solve needs tol / rel at most; half of that leaves room
// for the FP32 rounding of the correction.  Never tighter than inner_tol.
__host__ __device__ inline double inner_tol_for(double inner_tol, double tol, double rel) {
  const double need = rel > 0.0 ? 0.5 * tol / rel : 0.0;
  return need > inner_tol ? need : inner_tol;
}

// Per-solver workspace size (bytes), excluding nothing: callers add nothing.
size_t ws_bytes_for(const hs_op* A, hs_solver s, hs_dtype dt, int maxit);

// Solver launchers (hs_kernels.cu / hs_gs.cu).  They fill `res` (iters,
// status, rel_res, restarts) and copy the history if hist != nullptr.
hs_status run_jacobi(const SolveArgs& a, hs_result* res, double* hist);
hs_status run_cg(const SolveArgs& a, hs_result* res, double* hist);
hs_status run_bicgstab(const SolveArgs& a, hs_result* res, double* hist);
hs_status run_cg_nb(const SolveArgs& a, hs_result* res, double* hist);
bool jacobi_tb_applies(const SolveArgs& a);
hs_status run_jacobi_tb(const SolveArgs& a, hs_result* res, double* hist);
hs_status run_gauss_seidel(const SolveArgs& a, hs_result* res, double* hist);
// 27-point operator: one step per point hyperplane i + 2j + 4k (hs_gs27.cu).
hs_status run_gauss_seidel27(const SolveArgs& a, hs_result* res, double* hist);
size_t gs27_progress_bytes(const hs_op* A);
hs_status run_spmv(const hs_op* A, hs_dtype dt, const void* x, void* y, cudaStream_t st);
hs_status run_residual_plain(const hs_op* A, hs_dtype dt, const void* b, const void* x, void* r, cudaStream_t st);
size_t vark_coef_bytes(const hs_op* A, hs_dtype dt);
// Fills D (diagonal, or its inverse when invert_diag), ax, ay, az in dtype dt
// from the operator's k.
// Launch helpers shared by the solver translation units.
hs_status launch_coop(const void* fn, int grid, int block, void** args, size_t smem, cudaStream_t st);
hs_status init_ctrl(const Common& cm, const hs_opts& o, cudaStream_t st);
hs_status finish_solve_pub(const SolveArgs& sa, const Common& cm, const void* D, const void* ax, const void* ay,
                           const void* az, void* rbuf, hs_result* res, double* hist, bool want_hist);

// Diagnostic kernels: one bounded wait each, on a condition that never comes
// true (hs_diag_wait_timeout).  `ctrl` is initialised, `words` zeroed.
hs_status diag_team_wait(Ctrl* ctrl, double* partials, cudaStream_t st);       // hs_kernels.cu
hs_status diag_gs_wait(Ctrl* ctrl, const unsigned* flag, cudaStream_t st);     // hs_gs.cu
hs_status diag_gs27_wait(Ctrl* ctrl, const unsigned long long* words, cudaStream_t st);   // hs_gs27.cu
hs_status diag_gs27p_wait(Ctrl* ctrl, unsigned long long* words, cudaStream_t st);         // hs_gs27.cu

// Options with defaults filled in and validated (false: invalid, error set).
bool merge_opts(const hs_opts* in, hs_opts* out);

hs_status setup_vark(const hs_op* A, hs_dtype dt, void* D, void* ax, void* ay, void* az, bool invert_diag,
                     cudaStream_t st);

int sm_count();

// FP32 CG on a 3-D diffusion operator with TMA-staged planes and
// coefficients formed from k (hs_cg32v.cu).  cg32v_eligible: the grid and the
// options allow it.  k_to_f32: k32 = (float) k of the operator.
bool cg32v_eligible(const hs_op* A, const hs_opts& o);
hs_status k_to_f32(const hs_op* A, float* k32, cudaStream_t st);
hs_status cg32v_core(const hs_op* A, const float* k32, const float* b, float* x, double tol, int maxit,
                     const Common& cm, float* r, float* p0, float* p1, float* w, const hs_opts& o, cudaStream_t st);
// Thread-local record of whether the last solve staged its stencil planes
// with TMA (hs_last_staging).
void set_last_staging(int v);

}  // namespace hs
