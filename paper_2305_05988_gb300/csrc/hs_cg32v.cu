// hs_cg32v.cu -- FP32 conjugate gradient on the variable-coefficient diffusion
// operator -div(k grad u), 3-D, with the stencil planes staged in shared
// memory by the Tensor Memory Accelerator.  It is the inner solve of
// mixed-precision refinement on diffusion problems (and the FP32 hs_cg on a
// diffusion operator), and runs the classical CG iteration of section 3.2.
//
// The FP32 passes are bound by HBM bandwidth and by how many bytes an SM keeps
// in flight; the register-prefetch tile engine (hs_stencil.cuh) keeps one
// plane of loads per thread in flight and reads four FP32 coefficient arrays
// (D, ax, ay, az: 16 B per node).  Here:
//   - the face coefficients kappa_f / h_d^2 with kappa_f = 2 k_i k_j / (k_i +
//     k_j) (a boundary face: k_i) are formed on the fly from k itself, 4 B
//     per node instead of 16;
//   - each block stages whole tile planes (a 32 x BY tile plus a one-node
//     ring, box x from 4 nodes left of the tile so that every copy starts on
//     a 16-byte boundary) of the vectors a pass reads into a ring of R
//     shared-memory slots with cp.async.bulk.tensor; completion is counted on
//     one mbarrier per slot.  One thread issues the copies several planes
//     ahead of the plane the block computes, so the bytes in flight per SM
//     do not cost registers.  Nodes outside the grid arrive as zeros (the
//     TMA fill value), which are the Dirichlet ghost values;
//   - the x update of iteration k rides on pass 1 of iteration k + 1, so the
//     elementwise pass 2 reads w and r and writes r only (float4 accesses).
// Per node and iteration: pass 1 reads r, p_old, k, x and writes p, w, x
// (28 B); pass 2 reads w, r and writes r (12 B).  Dot products are
// accumulated in FP64 from exactly widened FP32 operands.
//
// Requirements (checked by cg32v_eligible): 3-D, n_x a multiple of 4 (row
// strides of the tensor maps are multiples of 16 bytes), n_x >= 40,
// n_y >= BY + 2, n_z >= 3, 16-byte aligned vectors.
#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "hs_krylov.cuh"

namespace hs {

namespace {

constexpr int TW = 32;               // tile width, one column per lane
constexpr int PADX = 4;              // box starts 4 nodes left of the tile
constexpr int BOXW = TW + 2 * PADX;  // 40 floats = 160 B per box row
#ifndef HS_TMA_SLOTS
#define HS_TMA_SLOTS 8
#endif
// ring slots: planes k-1, k, k+1 resident and NSLOT - 3 planes in flight; a
// power of two so that slot and phase of a stream position are bit fields
constexpr int NSLOT = HS_TMA_SLOTS;
constexpr int NSLOT_LOG2 = NSLOT == 4 ? 2 : NSLOT == 8 ? 3 : NSLOT == 16 ? 4 : -1;
static_assert(NSLOT_LOG2 > 0, "NSLOT must be 4, 8 or 16");

template <int BY>
struct Lay {
  static constexpr int HB = BOXW * (BY + 2) * 4;         // halo box bytes
  static constexpr int HBA = (HB + 127) & ~127;
  static constexpr int OB = TW * BY * 4;                 // owned box bytes
  static constexpr int OBA = (OB + 127) & ~127;
  static constexpr int SLOT = 3 * HBA + OBA;             // <= 3 halo boxes + 1 owned
  // ring, then the "full" and "empty" mbarriers of every slot
  static constexpr int BYTES = 128 + NSLOT * SLOT + 16 * NSLOT;
};

// ---- PTX wrappers: mbarrier and TMA ----------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Generic-proxy accesses of shared memory before async-proxy writes to it.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Generic-proxy global stores before async-proxy (TMA) reads of them.
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, unsigned long long* bar, int x, int y,
                                            int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

}  // namespace

struct Cg32vArgs {
  // tensor maps: halo boxes (BOXW x (BY+2) x 1) of r, p0, p1, k, x and owned
  // boxes (TW x BY x 1) of x and b
  CUtensorMap m_r, m_p[2], m_k, m_xh, m_xo, m_bo;
  Geom g;
  Tiling tl;
  float ihx, ihy, ihz;
  const float* b;
  float* x;
  float* r;
  float* p[2];
  float* w;
  Common cm;
  int maxit;
  double tol;
};

namespace {

enum { MODE_RESID = 0, MODE_P0 = 1, MODE_P = 2 };

// The block: BY compute warps (one tile row each) and one producer warp whose
// lane 0 issues the plane copies.  Slot s of the ring has a "full" mbarrier
// (one arrival by the producer plus the copied bytes) and an "empty" mbarrier
// (one arrival per compute warp when it is done with the slot's plane).
// Stream position q of the block (counted over all passes of the launch) uses
// slot q mod NSLOT for the (q div NSLOT)-th time: consumers wait on the full
// barrier with parity (q div NSLOT) mod 2, the producer waits on the empty
// barrier of the slot's previous use before re-arming it.  No block-wide
// barrier runs inside a pass.
template <int BY>
struct Engine {
  using L = Lay<BY>;
  unsigned char* ring;             // NSLOT slots, 128-byte aligned
  unsigned long long* full;        // NSLOT mbarriers
  unsigned long long* empty;       // NSLOT mbarriers
  const Cg32vArgs* a;
  const Team* tm;
  unsigned cnt;                    // stream positions of earlier passes

  __device__ __forceinline__ unsigned char* slot_ptr(unsigned q) const {
    return ring + (q & (NSLOT - 1)) * L::SLOT;
  }
  __device__ __forceinline__ const float* hbox(unsigned q, int k) const {
    return reinterpret_cast<const float*>(slot_ptr(q) + k * L::HBA);
  }
  __device__ __forceinline__ const float* obox(unsigned q) const {
    return reinterpret_cast<const float*>(slot_ptr(q) + 3 * L::HBA);
  }
  // Bounded wait for a phase of an mbarrier; false if the wait ran out or
  // another block reported an error.
  __device__ bool wait(unsigned long long* bar, unsigned parity) const {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    unsigned spins = 0;
    while (!mbar_try_wait(bar, parity)) {
      if ((++spins & 255u) == 0) {
        if (global_ns() - t0 > tm->ctrl->timeout_ns) return false;
        if (ld_acquire_int(&tm->ctrl->status) < 0) return false;
      }
    }
    return true;
  }
  __device__ __forceinline__ bool wait_full(unsigned q) const {
    return wait(full + (q & (NSLOT - 1)), (q >> NSLOT_LOG2) & 1u);
  }
};

__device__ __forceinline__ void item_planes(const Cg32vArgs& a, int item, int& i0, int& j0, int& z0, int& z1, int& qlo,
                                            int& qhi) {
  decode_item(a.tl, a.g, item, i0, j0, z0, z1);
  qlo = max(z0 - 1, 0);
  qhi = min(z1, a.g.nz - 1);
}

// One stencil pass over this block's work items: the producer warp issues the
// copies, the compute warps consume them.  Every thread returns whether the
// pass completed (false: a wait ran out or another block reported an error;
// the caller agrees block-wide and drains).  Returns the number of stream
// positions the pass used in *npos (identical in every thread).
template <int BY, int MODE>
__device__ bool tma_pass(const Engine<BY>& E, const float beta, const float ap, const float* pold, float* pnew,
                         double (&acc)[2], unsigned* npos) {
  using L = Lay<BY>;
  const Cg32vArgs& a = *E.a;
  const Team& tm = *E.tm;
  const Geom& g = a.g;
  const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
  const long long P = g.plane;
  // staged boxes: 0 = stencil source (x or r), 1 = k, 2 = p_old (MODE_P);
  // owned box: b (MODE_RESID) or x (MODE_P)
  constexpr int NH = MODE == MODE_P ? 3 : 2;
  constexpr int NO = MODE == MODE_P0 ? 0 : 1;
  constexpr unsigned BYTES = NH * L::HB + NO * L::OB;
  const int nitems = a.tl.items();
  // stream positions of this pass (the same count in every thread)
  unsigned total = 0;
  for (int item = tm.rank; item < nitems; item += tm.size) {
    int i0, j0, z0, z1, qlo, qhi;
    item_planes(a, item, i0, j0, z0, z1, qlo, qhi);
    total += (unsigned)(qhi - qlo + 1);
  }
  *npos = total;
  bool ok = true;

  if (ly == BY) {
    // ---- producer warp: lane 0 issues every position of the pass in order
    if (lx == 0) {
      const CUtensorMap* hm0 = MODE == MODE_RESID ? &a.m_xh : &a.m_r;
      const CUtensorMap* hm2 = pold == a.p[0] ? &a.m_p[0] : &a.m_p[1];
      const CUtensorMap* om = MODE == MODE_RESID ? &a.m_bo : &a.m_xo;
      unsigned q = 0;
      for (int item = tm.rank; item < nitems && ok; item += tm.size) {
        int i0, j0, z0, z1, qlo, qhi;
        item_planes(a, item, i0, j0, z0, z1, qlo, qhi);
        for (int z = qlo; z <= qhi; z++, q++) {
          const unsigned qa = E.cnt + q;
          const unsigned slot = qa & (NSLOT - 1), use = qa >> NSLOT_LOG2;
          // the slot's previous plane must have been released by every
          // compute warp
          if (use > 0 && !E.wait(E.empty + slot, (use - 1) & 1u)) {
            ok = false;
            break;
          }
          fence_proxy_async_smem();
          unsigned long long* bar = E.full + slot;
          unsigned char* sp = E.slot_ptr(qa);
          mbar_arrive_expect_tx(bar, BYTES);
          tma_load_3d(sp, hm0, bar, i0 - PADX, j0 - 1, z);
          tma_load_3d(sp + L::HBA, &a.m_k, bar, i0 - PADX, j0 - 1, z);
          if (NH == 3) tma_load_3d(sp + 2 * L::HBA, hm2, bar, i0 - PADX, j0 - 1, z);
          if (NO == 1) tma_load_3d(sp + 3 * L::HBA, om, bar, i0, j0, z);
        }
      }
      if (!ok) atomicCAS(&tm.ctrl->status, 0, (int)DS_TIMEOUT);
      // no copy of this block may still be in flight when the pass ends (or
      // the kernel gives up): wait (bounded) for the last ones issued
      const unsigned long long t0 = global_ns();
      for (unsigned d = q > (unsigned)NSLOT ? q - NSLOT : 0u; d < q; d++) {
        const unsigned qa = E.cnt + d;
        while (!mbar_try_wait(E.full + qa % NSLOT, (qa / NSLOT) & 1u)) {
          if (global_ns() - t0 > 2000000000ull) {
            ok = false;
            break;
          }
        }
      }
    }
    return ok;
  }

  // ---- compute warps
  const float fx = 2.0f * a.ihx, fy = 2.0f * a.ihy, fz = 2.0f * a.ihz;
  // face coefficient kappa / h^2 = 2 k_c k_n / (k_c + k_n) / h^2 (symmetric in
  // k_c, k_n bit for bit); a boundary face: k_c / h^2
  auto face = [](float kc, float kn, float f2) { return __fdividef((kc * kn) * f2, kc + kn); };
  auto release = [&](unsigned q) {
    __syncwarp();
    if (lx == 0) mbar_arrive(E.empty + (q & (NSLOT - 1)));
  };
  unsigned base = E.cnt;   // stream position of the current item's first plane
  for (int item = tm.rank; item < nitems; item += tm.size) {
    int i0, j0, z0, z1, qlo, qhi;
    item_planes(a, item, i0, j0, z0, z1, qlo, qhi);
    const int i = i0 + lx, j = j0 + ly;
    const bool inside = i < g.nx && j < g.ny;
    const bool hW = i > 0, hE = i + 1 < g.nx, hS = j > 0, hN = j + 1 < g.ny;
    const int cpos = (ly + 1) * BOXW + lx + PADX;    // own node in a halo box
    const int opos = ly * TW + lx;                    // own node in an owned box
    // stream positions and slot bases of planes z - 1, z, z + 1
    unsigned qz = base + (unsigned)(z0 - qlo);
    const float* Sb = nullptr;
    const float* Sc = reinterpret_cast<const float*>(E.slot_ptr(qz));
    // own stencil inputs of planes z - 1, z, z + 1 (zero outside the grid)
    float vb = 0.0f, vc, vt;
    auto src = [&](const float* S, int pos) -> float {
      const float v0 = S[pos];
      if constexpr (MODE == MODE_P) return fmaf(beta, S[2 * (L::HBA / 4) + pos], v0);
      return v0;
    };
    if (z0 - 1 >= 0) {
      ok &= E.wait_full(qz - 1);
      Sb = reinterpret_cast<const float*>(E.slot_ptr(qz - 1));
      vb = src(Sb, cpos);
    }
    ok &= E.wait_full(qz);
    vc = src(Sc, cpos);
    long long idx = (long long)j * g.nx + i + (long long)z0 * P;
    for (int z = z0; z < z1; z++, qz++, idx += P) {
      const float* St = nullptr;
      vt = 0.0f;
      if (z + 1 <= g.nz - 1) {
        ok &= E.wait_full(qz + 1);
        St = reinterpret_cast<const float*>(E.slot_ptr(qz + 1));
        vt = src(St, cpos);
      }
      if (inside && HS_IN_BOUNDS(idx, g.N)) {
        const float* K0 = Sc + L::HBA / 4;
        const float kc = K0[cpos];
        const float fW = hW ? face(kc, K0[cpos - 1], fx) : kc * a.ihx;
        const float fE = hE ? face(kc, K0[cpos + 1], fx) : kc * a.ihx;
        const float fS = hS ? face(kc, K0[cpos - BOXW], fy) : kc * a.ihy;
        const float fN = hN ? face(kc, K0[cpos + BOXW], fy) : kc * a.ihy;
        const float fB = (z > 0) ? face(kc, Sb[L::HBA / 4 + cpos], fz) : kc * a.ihz;
        const float fT = (z + 1 < g.nz) ? face(kc, St[L::HBA / 4 + cpos], fz) : kc * a.ihz;
        const float d = ((fW + fE) + (fS + fN)) + (fB + fT);
        float y = d * vc;
        y = fmaf(-fW, src(Sc, cpos - 1), y);
        y = fmaf(-fE, src(Sc, cpos + 1), y);
        y = fmaf(-fS, src(Sc, cpos - BOXW), y);
        y = fmaf(-fN, src(Sc, cpos + BOXW), y);
        y = fmaf(-fB, vb, y);
        y = fmaf(-fT, vt, y);
        if constexpr (MODE == MODE_RESID) {
          const float bv = Sc[3 * (L::HBA / 4) + opos];
          const float rv = bv - y;
          a.r[idx] = rv;
          acc[0] += widen(rv) * widen(rv);
          acc[1] += widen(bv) * widen(bv);
        } else {
          pnew[idx] = vc;
          a.w[idx] = y;
          acc[0] += widen(vc) * widen(y);
          if constexpr (MODE == MODE_P) {
            // the previous iteration's step x += alpha p_old
            a.x[idx] = fmaf(ap, Sc[2 * (L::HBA / 4) + cpos], Sc[3 * (L::HBA / 4) + opos]);
          }
        }
      }
      // this warp is done with plane z - 1 (ok is made warp-uniform first:
      // the lanes of a warp leave the loop together)
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      if (z - 1 >= qlo) release(qz - 1);
      vb = vc;
      vc = vt;
      Sb = Sc;
      Sc = St;
    }
    if (!ok) break;
    // planes z1 - 1 and z1 (if staged) are done too
    const unsigned qend = base + (unsigned)(z1 - 1 - qlo);
    release(qend);
    if (z1 <= qhi) release(qend + 1);
    base += (unsigned)(qhi - qlo + 1);
  }
  return ok;
}

}  // namespace

// Three resident blocks per SM: BY compute warps and one producer warp.
#ifndef HS_CG32V_MINB
#define HS_CG32V_MINB 3
#endif
template <int BY>
__global__ void __launch_bounds__(32 * (BY + 1), HS_CG32V_MINB) k_cg32v(const __grid_constant__ Cg32vArgs a) {
  using L = Lay<BY>;
  extern __shared__ unsigned char smraw[];
  __shared__ double sh[32 * MAX_SCAL];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smraw + 127) & ~(uintptr_t)127);
  const Team tm = grid_team(a.cm.ctrl, a.cm.partials);
  Engine<BY> E;
  E.ring = base;
  E.full = reinterpret_cast<unsigned long long*>(base + NSLOT * L::SLOT);
  E.empty = E.full + NSLOT;
  E.a = &a;
  E.tm = &tm;
  E.cnt = 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NSLOT; s++) {
      mbar_init(E.full + s, 1);
      mbar_init(E.empty + s, BY);
    }
    mbar_init_fence();
  }
  __syncthreads();
  const long long N = a.g.N;
  const long long st = tm.stride();

  // r = b - A x ; ||r||^2, ||b||^2
  double acc[2] = {0.0, 0.0};
  unsigned npos = 0;
  bool ok = tma_pass<BY, MODE_RESID>(E, 0.0f, 0.0f, a.p[0], nullptr, acc, &npos);
  // generic stores of a pass are read by TMA in later passes
  fence_proxy_async_global();
  if (!__syncthreads_and(ok)) return;
  E.cnt += npos;
  block_sum<2>(acc, sh);
  double s2[2];
  if (!team_reduce<2>(tm, acc, s2, sh)) return;
  double rr = s2[0];
  const double bb = s2[1];
  if (bb == 0.0) {
    for (long long q = tm.tid(); q < N; q += st) a.x[q] = 0.0f;
    if (tm.lead() && a.cm.hist) a.cm.hist[0] = 0.0;
    team_finish(tm, DS_CONVERGED, 0, 0.0);
    return;
  }
  double rel = sqrt(rr / bb);
  if (tm.lead() && a.cm.hist) a.cm.hist[0] = rel;
  if (rel <= a.tol || a.maxit == 0) {
    team_finish(tm, rel <= a.tol ? DS_CONVERGED : DS_MAXIT, 0, rel);
    return;
  }
  double beta = 0.0, alpha_prev = 0.0;
  int it = 0, status = DS_MAXIT;
  const long long N4 = N >> 2;
  float4* r4 = reinterpret_cast<float4*>(a.r);
  const float4* w4 = reinterpret_cast<const float4*>(a.w);
  while (it < a.maxit) {
    it++;
    float* pold = a.p[(it + 1) & 1];
    float* pnew = a.p[it & 1];
    // ---- pass 1: p = r + beta p_old ; w = A p ; p.w ; x += alpha_prev p_old
    double pw_acc[2] = {0.0, 0.0};
    ok = (it == 1) ? tma_pass<BY, MODE_P0>(E, 0.0f, 0.0f, pold, pnew, pw_acc, &npos)
                   : tma_pass<BY, MODE_P>(E, (float)beta, (float)alpha_prev, pold, pnew, pw_acc, &npos);
    fence_proxy_async_global();
    if (!__syncthreads_and(ok)) return;
    E.cnt += npos;
    double pw1[1] = {pw_acc[0]}, pw[1];
    block_sum<1>(pw1, sh);
    if (!team_reduce<1>(tm, pw1, pw, sh)) return;
    if (!(pw[0] > 0.0) || !isfinite(pw[0])) {
      status = isfinite(pw[0]) ? DS_BREAKDOWN : DS_NONFINITE;
      team_finish(tm, status, it, rel);   // x holds x_{it-1}
      return;
    }
    const double ar = rr / pw[0];
    const float tar = (float)ar;
    // ---- pass 2: r -= alpha w ; r.r
    double acc1[1] = {0.0};
    long long q = tm.tid();
    for (; q + st < N4; q += 2 * st) {
      float4 wa = __ldcg(w4 + q), wb = __ldcg(w4 + q + st);
      float4 ra = __ldcg(r4 + q), rb = __ldcg(r4 + q + st);
      ra.x = fmaf(-tar, wa.x, ra.x); ra.y = fmaf(-tar, wa.y, ra.y);
      ra.z = fmaf(-tar, wa.z, ra.z); ra.w = fmaf(-tar, wa.w, ra.w);
      rb.x = fmaf(-tar, wb.x, rb.x); rb.y = fmaf(-tar, wb.y, rb.y);
      rb.z = fmaf(-tar, wb.z, rb.z); rb.w = fmaf(-tar, wb.w, rb.w);
      r4[q] = ra;
      r4[q + st] = rb;
      acc1[0] += widen(ra.x) * widen(ra.x) + widen(ra.y) * widen(ra.y);
      acc1[0] += widen(ra.z) * widen(ra.z) + widen(ra.w) * widen(ra.w);
      acc1[0] += widen(rb.x) * widen(rb.x) + widen(rb.y) * widen(rb.y);
      acc1[0] += widen(rb.z) * widen(rb.z) + widen(rb.w) * widen(rb.w);
    }
    for (; q < N4; q += st) {
      float4 wa = __ldcg(w4 + q), ra = __ldcg(r4 + q);
      ra.x = fmaf(-tar, wa.x, ra.x); ra.y = fmaf(-tar, wa.y, ra.y);
      ra.z = fmaf(-tar, wa.z, ra.z); ra.w = fmaf(-tar, wa.w, ra.w);
      r4[q] = ra;
      acc1[0] += widen(ra.x) * widen(ra.x) + widen(ra.y) * widen(ra.y);
      acc1[0] += widen(ra.z) * widen(ra.z) + widen(ra.w) * widen(ra.w);
    }
    fence_proxy_async_global();
    block_sum<1>(acc1, sh);
    double rn[1];
    if (!team_reduce<1>(tm, acc1, rn, sh)) return;
    alpha_prev = ar;
    rel = sqrt(rn[0] / bb);
    if (tm.lead() && a.cm.hist) a.cm.hist[it] = rel;
    if (!isfinite(rel)) {
      status = DS_NONFINITE;
      break;
    }
    if (rel <= a.tol) {
      status = DS_CONVERGED;
      break;
    }
    beta = rn[0] / rr;
    rr = rn[0];
  }
  // the last step of x, x += alpha p_it
  {
    const float tax = (float)alpha_prev;
    const float* plast = a.p[it & 1];
    for (long long q = tm.tid(); q < N; q += st) a.x[q] = fmaf(tax, __ldcg(plast + q), __ldcg(a.x + q));
  }
  team_finish(tm, status, it, rel);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// A 3-D FP32 tensor map over an N-vector laid out as nz planes of ny rows of
// nx values, box (boxw, boxh, 1), zero fill outside the grid.
bool make_map(CUtensorMap* m, const void* base, const Geom& g, int boxw, int boxh) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || ((uintptr_t)base & 15u)) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
  const cuuint64_t strides[2] = {(cuuint64_t)g.nx * 4, (cuuint64_t)g.plane * 4};
  const cuuint32_t box[3] = {(cuuint32_t)boxw, (cuuint32_t)boxh, 1};
  const cuuint32_t es[3] = {1, 1, 1};
#ifndef HS_TMA_L2PROMO
#define HS_TMA_L2PROMO 2
#endif
  const CUtensorMapL2promotion promo = HS_TMA_L2PROMO == 0   ? CU_TENSOR_MAP_L2_PROMOTION_NONE
                                       : HS_TMA_L2PROMO == 1 ? CU_TENSOR_MAP_L2_PROMOTION_L2_128B
                                                             : CU_TENSOR_MAP_L2_PROMOTION_L2_256B;
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, promo,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

constexpr int CG32V_BY = 8;

}  // namespace

bool cg32v_eligible(const hs_op* A, const hs_opts&) {
  if (A->kind != KIND_DIFFUSION || A->ndim != 3) return false;
  const Geom g = geom_of(A);
  if (g.nx % 4 != 0 || g.nx < BOXW || g.ny < CG32V_BY + 2 || g.nz < 3) return false;
  return encode_fn() != nullptr;
}

__global__ void k_k_to_f32(const double* __restrict__ k, float* __restrict__ k32, long long N) {
  for (long long i = gtid(); i < N; i += gstride()) k32[i] = (float)k[i];
}

hs_status k_to_f32(const hs_op* A, float* k32, cudaStream_t st) {
  const Geom g = geom_of(A);
  const int blocks = (int)std::max<long long>(1, std::min<long long>((g.N + 255) / 256, (long long)sm_count() * 8));
  if (A->kdt == HS_F64) {
    k_k_to_f32<<<blocks, 256, 0, st>>>((const double*)A->k, k32, g.N);
  } else {
    cudaError_t e = cudaMemcpyAsync(k32, A->k, sizeof(float) * (size_t)g.N, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "k copy");
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HS_OK : cuda_fail(e, "k conversion launch");
}

hs_status cg32v_core(const hs_op* A, const float* k32, const float* b, float* x, double tol, int maxit,
                     const Common& cm, float* r, float* p0, float* p1, float* w, const hs_opts& o, cudaStream_t st) {
  constexpr int BY = CG32V_BY;
  using L = Lay<BY>;
  Cg32vArgs a;
  memset(&a, 0, sizeof(a));
  a.g = geom_of(A);
  a.ihx = (float)(1.0 / (A->h[0] * A->h[0]));
  a.ihy = (float)(1.0 / (A->h[1] * A->h[1]));
  a.ihz = (float)(1.0 / (A->h[2] * A->h[2]));
  a.b = b;
  a.x = x;
  a.r = r;
  a.p[0] = p0;
  a.p[1] = p1;
  a.w = w;
  a.cm = cm;
  a.maxit = maxit;
  a.tol = tol;
  const Geom& g = a.g;
  bool ok = make_map(&a.m_r, r, g, BOXW, BY + 2) && make_map(&a.m_p[0], p0, g, BOXW, BY + 2) &&
            make_map(&a.m_p[1], p1, g, BOXW, BY + 2) && make_map(&a.m_k, k32, g, BOXW, BY + 2) &&
            make_map(&a.m_xh, x, g, BOXW, BY + 2) && make_map(&a.m_xo, x, g, TW, BY) &&
            make_map(&a.m_bo, b, g, TW, BY);
  if (!ok) {
    set_error("tensor map encoding failed for the TMA-staged FP32 CG");
    return HS_ERR_INVALID;
  }
  hs_status s = init_ctrl(cm, o, st);
  if (s != HS_OK) return s;
  const size_t smem = L::BYTES;
  cudaError_t e = cudaFuncSetAttribute(k_cg32v<BY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "shared memory attribute");
  int grid = 0;
  s = plan_persistent(k_cg32v<BY>, 32 * (BY + 1), smem, g, BY, true, &grid, &a.tl, o, 1);
  if (s != HS_OK) return s;
  void* args[] = {&a};
  s = launch_coop((const void*)k_cg32v<BY>, grid, 32 * (BY + 1), args, smem, st);
  if (s != HS_OK) return s;
  return hs_dbg_take(st);
}

}  // namespace hs
