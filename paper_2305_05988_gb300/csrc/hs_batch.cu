// hs_batch.cu -- many independent systems solved by one persistent
// cooperative kernel, optionally replayed as a CUDA graph.
//
// Each system is solved by a team of blocks running the same CG / BiCGStab
// iteration bodies as the standalone solvers, with its own control block
// (team barrier, reduced scalars, status).  The host scheduler sizes teams by
// estimated work: a system whose work exceeds the planned makespan gets a team
// of several blocks that serves it alone; the remaining systems form a queue,
// largest first, that every block drains one system at a time once its team
// job (if any) is done.  A team's blocks therefore never wait for a block that
// is busy with another system, and converged systems stop taking block time.
//
// A batch whose systems all name HS_SOLVER_MIXED runs the mixed-precision
// kernel of hs_batch_mixed.cu instead (same plan, tables and graph cache).
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <mutex>
#include <new>
#include <numeric>
#include <vector>

#include "hs_batch.cuh"

namespace hs {

enum BatchKind : int {
  BK_CG_SYM2 = 0,
  BK_CG_SYM3,
  BK_CG_VARK2,
  BK_CG_VARK3,
  BK_BI_SYM2,
  BK_BI_SYM3,
  BK_BI_NONSYM2,
  BK_BI_NONSYM3,
  BK_BI_VARK2,
  BK_BI_VARK3,
};

struct BatchSys {
  int kind;
  int pad[3];
  CgArgs<double> cg;
  BiArgs<double> bi;
};
static_assert(sizeof(BatchSys) % 8 == 0, "descriptor must be copied in 8-byte words");


__device__ __forceinline__ Ctrl* sys_ctrl(const BatchSys& d) { return d.kind < BK_BI_SYM2 ? d.cg.cm.ctrl : d.bi.cm.ctrl; }
__device__ __forceinline__ double* sys_partials(const BatchSys& d) {
  return d.kind < BK_BI_SYM2 ? d.cg.cm.partials : d.bi.cm.partials;
}

__global__ void k_batch_init(const BatchSys* __restrict__ sys, int nsys, unsigned long long timeout_ns, int* head) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *head = 0;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsys; s += gridDim.x * blockDim.x) {
    Ctrl* c = sys_ctrl(sys[s]);
    c->count = 0;
    c->gen = 0;
    c->status = 0;
    c->iters = 0;
    c->restarts = 0;
    c->timeout_ns = timeout_ns;
    c->rel_res = -1.0;
  }
}

// Per-system outcome: status, iterations, relative residual, restarts.
__global__ void k_batch_gather(const BatchSys* __restrict__ sys, int nsys, double* __restrict__ out) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsys; s += gridDim.x * blockDim.x) {
    const Ctrl* c = sys_ctrl(sys[s]);
    double* o = out + (size_t)BATCH_OUT * s;
    o[0] = (double)c->status;
    o[1] = (double)c->iters;
    o[2] = c->rel_res;
    o[3] = (double)c->restarts;
    o[4] = 0.0;
    o[5] = 0.0;
  }
}

// Runs one job: stage the system's descriptor in shared memory and run its
// iteration body with the given team.
__device__ __forceinline__ void batch_job(const BatchSys* __restrict__ sys, int s, int rank, int size, BatchSys& d,
                                          double* sm, double* sh) {
  {
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(sys + s);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(&d);
    for (int w = threadIdx.x; w < (int)(sizeof(BatchSys) / 8); w += blockDim.x) dst[w] = src[w];
  }
  __syncthreads();
  Team tm;
  tm.rank = rank;
  tm.size = size;
  tm.ctrl = sys_ctrl(d);
  tm.partials = sys_partials(d);
  switch (d.kind) {
    case BK_CG_SYM2: team_finish(tm, cg_body<double, OP_SYM, 2, BATCH_CX>(d.cg, tm, sm, sh)); break;
    case BK_CG_SYM3: team_finish(tm, cg_body<double, OP_SYM, 3, BATCH_CX>(d.cg, tm, sm, sh)); break;
    case BK_CG_VARK2: team_finish(tm, cg_body<double, OP_VARK, 2, BATCH_CX>(d.cg, tm, sm, sh)); break;
    case BK_CG_VARK3: team_finish(tm, cg_body<double, OP_VARK, 3, BATCH_CX>(d.cg, tm, sm, sh)); break;
    case BK_BI_SYM2: team_finish(tm, bicgstab_body<double, OP_SYM, 2, BATCH_CX>(d.bi, tm, sm, sh)); break;
    case BK_BI_SYM3: team_finish(tm, bicgstab_body<double, OP_SYM, 3, BATCH_CX>(d.bi, tm, sm, sh)); break;
    case BK_BI_NONSYM2: team_finish(tm, bicgstab_body<double, OP_NONSYM, 2, BATCH_CX>(d.bi, tm, sm, sh)); break;
    case BK_BI_NONSYM3: team_finish(tm, bicgstab_body<double, OP_NONSYM, 3, BATCH_CX>(d.bi, tm, sm, sh)); break;
    case BK_BI_VARK2: team_finish(tm, bicgstab_body<double, OP_VARK, 2, BATCH_CX>(d.bi, tm, sm, sh)); break;
    default: team_finish(tm, bicgstab_body<double, OP_VARK, 3, BATCH_CX>(d.bi, tm, sm, sh)); break;
  }
  __syncthreads();
}

// Block b first runs its team job (if any: team blocks serve one large
// system each), then takes single-block systems from a queue ordered
// largest first until the queue is empty.  Queue jobs never wait on another
// block, so no block can wait on a block that is busy elsewhere.
__global__ void __launch_bounds__(BATCH_THREADS, HS_BATCH_MINBLOCKS) k_batch(const BatchSys* __restrict__ sys,
                                                         const int* __restrict__ job_off,
                                                         const BatchJob* __restrict__ jobs,
                                                         const int* __restrict__ queue, int nqueue,
                                                         int* __restrict__ head) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double sh[32 * MAX_SCAL];
  __shared__ BatchSys d;
  __shared__ int s_next;
  double* sm = reinterpret_cast<double*>(smraw);
  for (int j = job_off[blockIdx.x]; j < job_off[blockIdx.x + 1]; j++) {
    const BatchJob jb = jobs[j];
    batch_job(sys, jb.sys, jb.rank, jb.size, d, sm, sh);
  }
  for (;;) {
    if (threadIdx.x == 0) s_next = atomicAdd(head, 1);
    __syncthreads();
    const int q = s_next;
    __syncthreads();
    if (q >= nqueue) break;
    batch_job(sys, queue[q], 0, 1, d, sm, sh);
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

struct BatchPlanSys {
  int kind;
  int solver;
  Geom g;
  double work;
  int team;
  Tiling tl;
};

}  // namespace hs

struct hs_batch {
  int nsys;
  std::vector<hs_op> ops;             // copies of the operators (k stays borrowed)
  std::vector<int> solvers;
  bool mixed = false;                 // every system uses FP64 refinement with an FP32 inner solve
  // plan (depends on the grid size of the batched kernel)
  int grid = 0;
  std::vector<hs::BatchPlanSys> plan;
  std::vector<int> job_off;
  std::vector<hs::BatchJob> jobs;
  std::vector<int> queue;             // single-block systems, largest first
  std::vector<int> tile_planes;       // per system, 0 = cost model
  std::vector<size_t> sys_off;        // workspace offset of each system
  size_t tables_bytes = 0;
  size_t ws_total = 0;
  // graph cache
  cudaGraphExec_t exec = nullptr;
  void* exec_ws = nullptr;
  cudaStream_t exec_stream = nullptr;
  int graph_used = 0;
  std::mutex mu;
};

namespace hs {

// Inner solver of a mixed-precision system: CG for the symmetric operators,
// BiCGStab for the upwind one.
static int mixed_inner(const hs_op* A) { return opkind_of(A) == OP_NONSYM ? HS_SOLVER_BICGSTAB : HS_SOLVER_CG; }

static int batch_kind(const hs_op* A, int solver) {
  const bool d3 = A->ndim >= 3;
  const int opk = opkind_of(A);
  if (solver == HS_SOLVER_MIXED) {
    if (mixed_inner(A) == HS_SOLVER_CG) {
      if (opk == OP_SYM) return d3 ? MK_CG_SYM3 : MK_CG_SYM2;
      return d3 ? MK_CG_VARK3 : MK_CG_VARK2;
    }
    if (opk == OP_SYM) return d3 ? MK_BI_SYM3 : MK_BI_SYM2;
    if (opk == OP_NONSYM) return d3 ? MK_BI_NONSYM3 : MK_BI_NONSYM2;
    return d3 ? MK_BI_VARK3 : MK_BI_VARK2;
  }
  if (solver == HS_SOLVER_CG) {
    if (opk == OP_SYM) return d3 ? BK_CG_SYM3 : BK_CG_SYM2;
    if (opk == OP_VARK) return d3 ? BK_CG_VARK3 : BK_CG_VARK2;
    return -1;
  }
  if (opk == OP_SYM) return d3 ? BK_BI_SYM3 : BK_BI_SYM2;
  if (opk == OP_NONSYM) return d3 ? BK_BI_NONSYM3 : BK_BI_NONSYM2;
  return d3 ? BK_BI_VARK3 : BK_BI_VARK2;
}

static size_t batch_smem() { return slab_bytes<double>(BATCH_BY, BATCH_CX); }

static int cx_of(int) { return BATCH_CX; }

static int batch_grid(bool mixed) {
  int per_sm = 0;
  if (mixed) {
    per_sm = batch_mx_blocks_per_sm(BATCH_THREADS, batch_smem());
  } else if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, BATCH_THREADS, batch_smem()) !=
             cudaSuccess) {
    per_sm = 0;
  }
  if (per_sm < 1) return 0;
  return std::min(per_sm * sm_count(), MAX_BLOCKS);
}

// Estimated solver work: unknowns x iterations x relative cost per
// iteration.  Iterations of CG on these operators grow like the grid side:
// about (n + 1) ln(2/tol) / (2 pi); BiCGStab needs ~0.65 as many iterations
// at ~2.2 times the cost.  A mixed-precision system does about as many
// inner iterations in all, at about half the cost each (FP32 arithmetic and
// half the bytes).
static double est_work(const hs_op* A, int solver, double tol) {
  double nmax = 1;
  for (int d = 0; d < A->ndim; d++) nmax = std::max(nmax, (double)A->n[d]);
  const double N = (double)(A->n[0] * A->n[1] * A->n[2]);
  const double it = std::max(2.0, (nmax + 1.0) * std::log(2.0 / std::max(tol, 1e-300)) / (2.0 * M_PI));
  if (solver == HS_SOLVER_MIXED) return 0.5 * est_work(A, mixed_inner(A), tol);
  return solver == HS_SOLVER_CG ? N * it : N * 0.65 * it * 2.2;
}

// Team sizes and job lists for `grid` blocks.  The makespan T is found by
// bisection: a system with work W > T gets a team of ceil(W/T) blocks, the
// rest go to the shared queue, and T is feasible when the teams leave enough
// blocks for the queued work at T per block.
static void make_plan(hs_batch* B, int grid, double tol) {
  const int n = B->nsys;
  B->plan.assign(n, BatchPlanSys{});
  double total = 0.0, wmax = 0.0;
  for (int s = 0; s < n; s++) {
    BatchPlanSys& p = B->plan[s];
    p.solver = B->solvers[s];
    p.kind = batch_kind(&B->ops[s], p.solver);
    p.g = geom_of(&B->ops[s]);
    p.work = est_work(&B->ops[s], p.solver, tol);
    p.team = 0;
    total += p.work;
    wmax = std::max(wmax, p.work);
  }
  auto team_cap = [&](const BatchPlanSys& p) {
    Tiling t1 = choose_tiling(p.g, BATCH_BY, 0, true, 0, cx_of(p.solver));
    return std::max(1, t1.tiles_x * t1.tiles_y * std::max(1, p.g.nz / 4));
  };
  auto blocks_needed = [&](double T) {
    double small = 0.0;
    long long teams = 0;
    for (const BatchPlanSys& p : B->plan) {
      if (p.work > T)
        teams += std::min<long long>(team_cap(p), (long long)std::ceil(p.work / T));
      else
        small += p.work;
    }
    return (double)teams + std::ceil(small / T);
  };
  double lo = total / grid, hi = std::max(wmax, total / grid) * 2.0;
  for (int it = 0; it < 60; it++) {
    const double mid = 0.5 * (lo + hi);
    if (blocks_needed(mid) <= grid) hi = mid;
    else lo = mid;
  }
  const double T = hi;
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int a, int b) { return B->plan[a].work > B->plan[b].work; });
  std::vector<std::vector<BatchJob>> per_block(grid);
  int next = 0;
  B->queue.clear();
  for (int s : order) {
    BatchPlanSys& p = B->plan[s];
    if (p.work > T && next < grid) {
      p.team = std::max(1, std::min({team_cap(p), (int)std::ceil(p.work / T), grid - next}));
      for (int r = 0; r < p.team; r++) per_block[next + r].push_back(BatchJob{s, r, p.team, 0});
      next += p.team;
    } else {
      p.team = 1;
      B->queue.push_back(s);   // largest first
    }
    p.tl = choose_tiling(p.g, BATCH_BY, p.team, true, B->tile_planes.empty() ? 0 : B->tile_planes[s],
                         cx_of(p.solver));
  }
  B->job_off.assign(grid + 1, 0);
  B->jobs.clear();
  for (int b = 0; b < grid; b++) {
    B->job_off[b] = (int)B->jobs.size();
    for (const BatchJob& j : per_block[b]) B->jobs.push_back(j);
  }
  B->job_off[grid] = (int)B->jobs.size();
  B->grid = grid;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Workspace: descriptor table, job tables, results, then per system a control
// block, its team's partial sums and its solver vectors (+ coefficients).
static size_t desc_bytes(const hs_batch* B) { return B->mixed ? sizeof(MxSys) : sizeof(BatchSys); }

// Vectors of a system: FP64 solver vectors, or for a mixed system the FP32
// residual and correction plus the inner solver's FP32 vectors.
static int sys_vectors(const hs_batch* B, int s) {
  const int solver = B->mixed ? mixed_inner(&B->ops[s]) : B->plan[s].solver;
  return (solver == HS_SOLVER_CG ? 4 : 8) + (B->mixed ? 2 : 0);
}

static void layout(hs_batch* B) {
  const int n = B->nsys;
  size_t off = 0;
  off += align256(desc_bytes(B) * n);
  off += align256(sizeof(int) * (B->grid + 1));
  off += align256(sizeof(BatchJob) * std::max<size_t>(1, B->jobs.size()));
  off += align256(sizeof(double) * BATCH_OUT * n);
  off += align256(sizeof(int) * (n + 1));   // queue + head
  B->tables_bytes = off;
  B->sys_off.assign(n, 0);
  for (int s = 0; s < n; s++) {
    const BatchPlanSys& p = B->plan[s];
    B->sys_off[s] = off;
    off += B->mixed ? 1024 : 512;           // control block(s)
    off += align256(sizeof(double) * MAX_SCAL * p.team);
    const size_t el = B->mixed ? sizeof(float) : sizeof(double);
    off += align256(el * (size_t)p.g.N) * sys_vectors(B, s);
    if (B->ops[s].kind == KIND_DIFFUSION) {
      off += 4 * align256(sizeof(double) * (size_t)p.g.N);
      if (B->mixed) off += 4 * align256(sizeof(float) * (size_t)p.g.N);
    }
  }
  B->ws_total = off;
}

// The plan is made once per batch: the work estimates use a nominal
// tolerance of 1e-8 (the tolerance only scales every estimate by the same
// logarithmic factor).
static hs_status ensure_plan(hs_batch* B) {
  if (B->grid > 0) return HS_OK;
  int grid = batch_grid(B->mixed);
  if (grid < 1) {
    set_error("batched kernel cannot be resident");
    return HS_ERR_CUDA;
  }
  make_plan(B, grid, 1e-8);
  layout(B);
  if (B->exec) {
    cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
  }
  return HS_OK;
}

// Descriptor of mixed-precision system s for one call: carves its control
// blocks and vectors from the workspace and sets up its coefficients.
static hs_status fill_mixed(hs_batch* B, int s, const double* b, double* x, double tol, int maxit, const hs_opts& o,
                            char* base, cudaStream_t stm, MxSys* out) {
  const hs_op* A = &B->ops[s];
  const BatchPlanSys& p = B->plan[s];
  Carve c{base + B->sys_off[s], 0, (size_t)-1, true};
  Common cm;
  cm.ctrl = c.take<Ctrl>(1);
  c.take<char>(512 - ((sizeof(Ctrl) + 255) & ~(size_t)255));
  Ctrl* inner = c.take<Ctrl>(1);
  c.take<char>(512 - ((sizeof(Ctrl) + 255) & ~(size_t)255));
  cm.partials = c.take<double>((size_t)MAX_SCAL * p.team);
  cm.hist = nullptr;
  const int nv = sys_vectors(B, s);
  float* v[10] = {nullptr};
  for (int q = 0; q < nv; q++) v[q] = c.take<float>(p.g.N);
  double *D = nullptr, *ax = nullptr, *ay = nullptr, *az = nullptr;
  float *D32 = nullptr, *ax32 = nullptr, *ay32 = nullptr, *az32 = nullptr;
  if (A->kind == KIND_DIFFUSION) {
    D = c.take<double>(p.g.N);
    ax = c.take<double>(p.g.N);
    ay = c.take<double>(p.g.N);
    az = c.take<double>(p.g.N);
    D32 = c.take<float>(p.g.N);
    ax32 = c.take<float>(p.g.N);
    ay32 = c.take<float>(p.g.N);
    az32 = c.take<float>(p.g.N);
    hs_status s2 = setup_vark(A, HS_F64, D, ax, ay, az, false, stm);
    if (s2 == HS_OK) s2 = setup_vark(A, HS_F32, D32, ax32, ay32, az32, false, stm);
    if (s2 != HS_OK) return s2;
  }
  MxSys& d = *out;
  memset(&d, 0, sizeof(d));
  d.kind = p.kind;
  d.max_outer = maxit;
  d.tol = tol;
  d.restart_eps = o.restart_eps;
  d.inner_tol = o.inner_tol;
  d.inner_fixed = o.inner_fixed_tol;
  d.g = p.g;
  d.tl = p.tl;
  d.cf = op_coef<double>(A, D, ax, ay, az, &d.sigma);
  d.b = b;
  d.x = x;
  d.r32 = v[0];
  d.d32 = v[1];
  d.cm = cm;
  d.inner_ctrl = inner;
  Common ci = cm;
  ci.ctrl = inner;
  double sig32 = 1.0;
  const Coef<float> cf32 = op_coef<float>(A, D32, ax32, ay32, az32, &sig32);
  if (mixed_inner(A) == HS_SOLVER_CG) {
    CgArgs<float>& a = d.cg;
    a.g = p.g;
    a.tl = p.tl;
    a.cf = cf32;
    a.sigma = sig32;
    a.b = d.r32;
    a.x = d.d32;
    a.r = v[2];
    a.p0 = v[3];
    a.p1 = v[4];
    a.w = v[5];
    a.cm = ci;
    a.maxit = o.inner_maxit;
    a.tol = o.inner_tol;
  } else {
    BiArgs<float>& a = d.bi;
    a.g = p.g;
    a.tl = p.tl;
    a.cf = cf32;
    a.sigma = sig32;
    a.b = d.r32;
    a.x = d.d32;
    a.r = v[2];
    a.rs = v[3];
    a.p0 = v[4];
    a.p1 = v[5];
    a.v0 = v[6];
    a.v1 = v[7];
    a.s = v[8];
    a.t = v[9];
    a.cm = ci;
    a.maxit = o.inner_maxit;
    a.tol = o.inner_tol;
    a.reps = o.restart_eps;   // rescaled on the device for each correction solve
  }
  return HS_OK;
}

}  // namespace hs

using namespace hs;

extern "C" hs_status hs_batch_create(int nsys, const hs_op* const* ops, const int* solvers, hs_batch** out) {
  if (!out) {
    set_error("out is NULL");
    return HS_ERR_INVALID;
  }
  *out = nullptr;
  if (nsys < 1 || !ops || !solvers) {
    set_error("batch needs nsys >= 1, ops and solvers");
    return HS_ERR_INVALID;
  }
  hs_batch* B = new (std::nothrow) hs_batch;
  if (!B) {
    set_error("out of host memory");
    return HS_ERR_INVALID;
  }
  B->nsys = nsys;
  B->ops.resize(nsys);
  B->solvers.resize(nsys);
  B->mixed = solvers[0] == HS_SOLVER_MIXED;
  for (int s = 0; s < nsys; s++) {
    if (!ops[s] || (solvers[s] != HS_SOLVER_CG && solvers[s] != HS_SOLVER_BICGSTAB && solvers[s] != HS_SOLVER_MIXED)) {
      set_error("system %d: operator missing or solver not CG / BiCGStab / mixed", s);
      delete B;
      return HS_ERR_INVALID;
    }
    if (opkind_of(ops[s]) == OP_BOX27) {
      set_error("system %d: the batched solver takes 7-point operators", s);
      delete B;
      return HS_ERR_INVALID;
    }
    if ((solvers[s] == HS_SOLVER_MIXED) != B->mixed) {
      set_error("system %d: a batch is either all mixed precision or all FP64", s);
      delete B;
      return HS_ERR_INVALID;
    }
    if (solvers[s] == HS_SOLVER_CG && opkind_of(ops[s]) == OP_NONSYM) {
      set_error("system %d: CG needs a symmetric operator", s);
      delete B;
      return HS_ERR_INVALID;
    }
    B->ops[s] = *ops[s];
    B->solvers[s] = solvers[s];
  }
  *out = B;
  return HS_OK;
}

extern "C" void hs_batch_destroy(hs_batch* B) {
  if (!B) return;
  if (B->exec) cudaGraphExecDestroy(B->exec);
  delete B;
}

extern "C" hs_status hs_batch_workspace_size(hs_batch* B, size_t* bytes) {
  if (!B || !bytes) {
    set_error("NULL argument");
    return HS_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lock(B->mu);
  hs_status s = ensure_plan(B);
  if (s != HS_OK) return s;
  *bytes = B->ws_total;
  return HS_OK;
}

extern "C" hs_status hs_batch_solve(hs_batch* B, const double* const* b, double* const* x, double tol, int maxit,
                                    const hs_opts* opts, void* ws, size_t ws_bytes, void* stream, hs_result* res) {
  hs::NvtxRange range("hs_batch_solve");
  if (!B || !b || !x || !res) {
    set_error("NULL argument");
    return HS_ERR_INVALID;
  }
  if (!(tol >= 0.0) || !std::isfinite(tol) || maxit < 0) {
    set_error("tol must be finite and >= 0, maxit >= 0");
    return HS_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lock(B->mu);
  hs_status st = ensure_plan(B);
  if (st != HS_OK) return st;
  if (!ws || ((uintptr_t)ws % 256) != 0 || ws_bytes < B->ws_total) {
    set_error("batch workspace missing, misaligned or too small (%zu < %zu)", ws_bytes, B->ws_total);
    return HS_ERR_WORKSPACE;
  }
  hs_opts o;
  if (!merge_opts(opts, &o)) return HS_ERR_INVALID;
  const double timeout_s = o.timeout_s;
  const int use_graph = o.use_graph;
  cudaStream_t stm = (cudaStream_t)stream;
  const int n = B->nsys;
  char* base = (char*)ws;
  void* d_sys = base;
  int* d_joboff = (int*)(base + align256(desc_bytes(B) * n));
  BatchJob* d_jobs = (BatchJob*)((char*)d_joboff + align256(sizeof(int) * (B->grid + 1)));
  double* d_out = (double*)((char*)d_jobs + align256(sizeof(BatchJob) * std::max<size_t>(1, B->jobs.size())));
  int* d_head = (int*)((char*)d_out + align256(sizeof(double) * BATCH_OUT * n));
  int* d_queue = d_head + 1;
  const int nqueue = (int)B->queue.size();
  // descriptors for this call (b, x pointers may change between calls)
  std::vector<BatchSys> hsys(B->mixed ? 0 : n);
  std::vector<MxSys> hmx(B->mixed ? n : 0);
  for (int s = 0; s < n; s++) {
    const hs_op* A = &B->ops[s];
    const BatchPlanSys& p = B->plan[s];
    if (!b[s] || !x[s] || ((uintptr_t)b[s] % 16) || ((uintptr_t)x[s] % 16)) {
      set_error("system %d: b and x must be 16-byte aligned device pointers", s);
      return HS_ERR_INVALID;
    }
    if (B->mixed) {
      hs_status sm = fill_mixed(B, s, b[s], x[s], tol, maxit, o, base, stm, &hmx[s]);
      if (sm != HS_OK) return sm;
      continue;
    }
    Carve c{base + B->sys_off[s], 0, (size_t)-1, true};
    Common cm;
    cm.ctrl = c.take<Ctrl>(1);
    c.take<char>(512 - ((sizeof(Ctrl) + 255) & ~(size_t)255));
    cm.partials = c.take<double>((size_t)MAX_SCAL * p.team);
    cm.hist = nullptr;
    BatchSys& d = hsys[s];
    memset(&d, 0, sizeof(d));
    d.kind = p.kind;
    const int nv = p.solver == HS_SOLVER_CG ? 4 : 8;
    double* v[8] = {nullptr};
    for (int q = 0; q < nv; q++) v[q] = c.take<double>(p.g.N);
    double *D = nullptr, *ax = nullptr, *ay = nullptr, *az = nullptr;
    if (A->kind == KIND_DIFFUSION) {
      D = c.take<double>(p.g.N);
      ax = c.take<double>(p.g.N);
      ay = c.take<double>(p.g.N);
      az = c.take<double>(p.g.N);
      hs_status s2 = setup_vark(A, HS_F64, D, ax, ay, az, false, stm);
      if (s2 != HS_OK) return s2;
    }
    double sigma = 1.0;
    Coef<double> cf = op_coef<double>(A, D, ax, ay, az, &sigma);
    if (p.solver == HS_SOLVER_CG) {
      CgArgs<double>& a = d.cg;
      a.g = p.g;
      a.tl = p.tl;
      a.cf = cf;
      a.sigma = sigma;
      a.b = b[s];
      a.x = x[s];
      a.r = v[0];
      a.p0 = v[1];
      a.p1 = v[2];
      a.w = v[3];
      a.cm = cm;
      a.maxit = maxit;
      a.tol = tol;
    } else {
      BiArgs<double>& a = d.bi;
      a.g = p.g;
      a.tl = p.tl;
      a.cf = cf;
      a.sigma = sigma;
      a.b = b[s];
      a.x = x[s];
      a.r = v[0];
      a.rs = v[1];
      a.p0 = v[2];
      a.p1 = v[3];
      a.v0 = v[4];
      a.v1 = v[5];
      a.s = v[6];
      a.t = v[7];
      a.cm = cm;
      a.maxit = maxit;
      a.tol = tol;
      a.reps = o.restart_eps;
    }
  }
  cudaError_t e = B->mixed ? cudaMemcpyAsync(d_sys, hmx.data(), sizeof(MxSys) * n, cudaMemcpyHostToDevice, stm)
                           : cudaMemcpyAsync(d_sys, hsys.data(), sizeof(BatchSys) * n, cudaMemcpyHostToDevice, stm);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_joboff, B->job_off.data(), sizeof(int) * (B->grid + 1), cudaMemcpyHostToDevice, stm);
  if (e == cudaSuccess && !B->jobs.empty())
    e = cudaMemcpyAsync(d_jobs, B->jobs.data(), sizeof(BatchJob) * B->jobs.size(), cudaMemcpyHostToDevice, stm);
  if (e == cudaSuccess && nqueue > 0)
    e = cudaMemcpyAsync(d_queue, B->queue.data(), sizeof(int) * nqueue, cudaMemcpyHostToDevice, stm);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stm);   // host tables go out of scope below
  if (e != cudaSuccess) return cuda_fail(e, "batch table upload");

  const unsigned long long tns = (unsigned long long)(timeout_s * 1e9);
  const int ib = std::max(1, std::min(64, (n + 255) / 256));
  const size_t smem = batch_smem();
  auto launch_all = [&](cudaStream_t s) -> cudaError_t {
    if (B->mixed)
      return batch_mx_launch(s, B->grid, smem, (const MxSys*)d_sys, n, tns, d_joboff, d_jobs, d_queue, nqueue, d_head,
                             d_out);
    k_batch_init<<<ib, 256, 0, s>>>((const BatchSys*)d_sys, n, tns, d_head);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(B->grid);
    cfg.blockDim = dim3(BATCH_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t le = cudaLaunchKernelEx(&cfg, k_batch, (const BatchSys*)d_sys, (const int*)d_joboff,
                                        (const BatchJob*)d_jobs, (const int*)d_queue, nqueue, d_head);
    if (le != cudaSuccess) return le;
    k_batch_gather<<<ib, 256, 0, s>>>((const BatchSys*)d_sys, n, d_out);
    return cudaGetLastError();
  };
  B->graph_used = 0;
  bool launched = false;
  if (use_graph && stm != nullptr) {
    if (!B->exec || B->exec_ws != ws || B->exec_stream != stm) {
      if (B->exec) {
        cudaGraphExecDestroy(B->exec);
        B->exec = nullptr;
      }
      cudaGraph_t graph = nullptr;
      e = cudaStreamBeginCapture(stm, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t le = launch_all(stm);
        e = cudaStreamEndCapture(stm, &graph);
        if (le != cudaSuccess) e = le;
      }
      if (e == cudaSuccess && graph) e = cudaGraphInstantiate(&B->exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        B->exec = nullptr;
        cudaGetLastError();   // capture not available: fall back to direct launches
      } else {
        B->exec_ws = ws;
        B->exec_stream = stm;
      }
    }
    if (B->exec) {
      e = cudaGraphLaunch(B->exec, stm);
      if (e != cudaSuccess) return cuda_fail(e, "batch graph launch");
      B->graph_used = 1;
      launched = true;
    }
  }
  if (!launched) {
    e = launch_all(stm);
    if (e != cudaSuccess) return cuda_fail(e, "batch launch");
  }
  std::vector<double> outh((size_t)BATCH_OUT * n);
  e = cudaMemcpyAsync(outh.data(), d_out, sizeof(double) * BATCH_OUT * n, cudaMemcpyDeviceToHost, stm);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stm);
  if (e != cudaSuccess) return cuda_fail(e, "batched solve");
  hs_status worst = HS_OK;
  for (int s = 0; s < n; s++) {
    const double* q = &outh[(size_t)BATCH_OUT * s];
    const int dsx = (int)q[0];
    hs_result& r = res[s];
    memset(&r, 0, sizeof(r));
    r.iters = (int)q[1];
    r.rel_res = q[2];
    r.true_rel_res = B->mixed ? q[2] : -1.0;   // a mixed system's residual is the FP64 b - A x
    r.restarts = (int)q[3];
    r.outer = (int)q[4];
    r.inner_iters = (long long)q[5];
    switch (dsx) {
      case DS_CONVERGED: r.status = HS_OK; break;
      case DS_MAXIT: r.status = HS_NOT_CONVERGED; break;
      case DS_BREAKDOWN: r.status = HS_ERR_BREAKDOWN; break;
      case DS_NONFINITE: r.status = HS_ERR_NONFINITE; break;
      case DS_TIMEOUT: r.status = HS_ERR_TIMEOUT; break;
      default: r.status = HS_ERR_CUDA; break;
    }
    if (r.status == HS_ERR_TIMEOUT || r.status == HS_ERR_CUDA) worst = (hs_status)r.status;
  }
  if (worst == HS_ERR_TIMEOUT) set_error("a device-side wait ran out in the batched solve");
  if (worst == HS_ERR_CUDA) set_error("a system of the batch ended without a status");
  return worst;
}

extern "C" hs_status hs_batch_set_tile_planes(hs_batch* B, const int* planes) {
  if (!B || !planes) {
    set_error("NULL argument");
    return HS_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lock(B->mu);
  B->tile_planes.assign(planes, planes + B->nsys);
  for (int& v : B->tile_planes) v = std::max(0, v);
  B->grid = 0;   // re-plan on next use
  if (B->exec) {
    cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
  }
  return HS_OK;
}

extern "C" int hs_batch_graph_used(const hs_batch* B) { return B ? B->graph_used : 0; }
extern "C" int hs_batch_grid(const hs_batch* B) { return B ? B->grid : 0; }
extern "C" hs_status hs_batch_team_sizes(const hs_batch* B, int* teams) {
  if (!B || !teams) {
    set_error("NULL argument");
    return HS_ERR_INVALID;
  }
  if (B->grid == 0) {
    set_error("batch not planned yet (call hs_batch_workspace_size first)");
    return HS_ERR_INVALID;
  }
  for (int s = 0; s < B->nsys; s++) teams[s] = B->plan[s].team;
  return HS_OK;
}
