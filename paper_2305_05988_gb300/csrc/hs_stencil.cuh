// hs_stencil.cuh -- the z-marching tile engine used by every stencil pass.
//
// A work item is an xy tile of BX x BY nodes (BX = 32, one warp per row) and
// a range [z0, z1) of planes.  The block marches up the planes: each thread
// keeps the values of its own column at planes k-1, k, k+1 in registers,
// while the plane k itself (tile plus a one-node halo) sits in a
// double-buffered shared-memory slab that supplies the W/E/S/N neighbours.
// One __syncthreads per plane.
//
// The stencil INPUT value at a node is produced by a functor `src` (a plain
// load for SpMV/Jacobi, or an on-the-fly vector update such as
// p = r + beta p for the Krylov passes); halo values are produced by whole
// warps (warp 0: row below, warp 1: row above, warp 2: the two side
// columns), so FP64 work is never issued for a handful of lanes.
// Nodes outside the grid read as zero (homogeneous Dirichlet ghosts).
#pragma once
#include "hs_common.cuh"

namespace hs {

constexpr int BX = 32;

struct Tiling {
  int by;        // rows per tile (3..16), blockDim.x = 32 * by
  int tiles_x, tiles_y, chunks, lz;
  __host__ __device__ int items() const { return tiles_x * tiles_y * chunks; }
};

// Decode a work item: consecutive items cover the tiles of one z chunk, so
// blocks running concurrently work on neighbouring planes (L2 reuse).
__device__ __forceinline__ void decode_item(const Tiling& t, const Geom& g, int item, int& i0, int& j0,
                                            int& z0, int& z1) {
  int txy = t.tiles_x * t.tiles_y;
  int c = item / txy;
  int r = item - c * txy;
  int ty = r / t.tiles_x;
  int tx = r - ty * t.tiles_x;
  i0 = tx * BX;
  j0 = ty * t.by;
  z0 = c * t.lz;
  z1 = min(g.nz, z0 + t.lz);
}

// Shared slab: 2 planes of (by + 2) x (BX + 2) values.
template <typename T>
__device__ __forceinline__ T& slab(T* sm, int by, int buf, int row, int col) {
  return sm[(buf * (by + 2) + row) * (BX + 2) + col];
}

// Fill the halo of plane kk into slab buffer `buf` (warps 0..2 only).
template <typename T, class Src>
__device__ __forceinline__ void fill_halo(const Geom& g, int by, T* sm, int buf, int i0, int j0, int kk,
                                          Src& src) {
  const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
  const long long pk = (long long)kk * g.plane;
  if (ly == 0) {
    int i = i0 + lx, j = j0 - 1;
    T v = T(0);
    if (j >= 0 && i < g.nx) v = src(pk + (long long)j * g.nx + i, false);
    slab(sm, by, buf, 0, lx + 1) = v;
  } else if (ly == 1) {
    int i = i0 + lx, j = j0 + by;
    T v = T(0);
    if (j < g.ny && i < g.nx) v = src(pk + (long long)j * g.nx + i, false);
    slab(sm, by, buf, by + 1, lx + 1) = v;
  } else if (ly == 2) {
    if (lx < by) {
      int i = i0 - 1, j = j0 + lx;
      T v = T(0);
      if (i >= 0 && j < g.ny) v = src(pk + (long long)j * g.nx + i, false);
      slab(sm, by, buf, lx + 1, 0) = v;
    } else if (lx >= 16 && lx < 16 + by) {
      int i = i0 + BX, j = j0 + lx - 16;
      T v = T(0);
      if (i < g.nx && j < g.ny) v = src(pk + (long long)j * g.nx + i, false);
      slab(sm, by, buf, lx - 16 + 1, BX + 1) = v;
    }
  }
}

// Neighbour values of the current node handed to the stencil functor.
template <typename T>
struct Nbr {
  T c, w, e, s, n, b, t;
};

// Process one work item.  `src(idx, own)` returns the stencil input at a
// node (own = the node belongs to this item, so side outputs may be stored);
// `sink(idx, nb, i, j, k)` consumes the neighbourhood of each owned node.
template <typename T, int NDIM, class Src, class Sink>
__device__ __forceinline__ void zmarch_item(const Geom& g, const Tiling& tl, int item, T* sm, Src& src,
                                            Sink& sink) {
  int i0, j0, z0, z1;
  decode_item(tl, g, item, i0, j0, z0, z1);
  const int by = tl.by;
  const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
  const int i = i0 + lx, j = j0 + ly;
  const bool inside = (i < g.nx) && (j < g.ny);
  const long long col = (long long)j * g.nx + i;

  T vb = T(0), vc = T(0), vt = T(0);
  if (NDIM == 3 && inside && z0 > 0) vb = src(col + (long long)(z0 - 1) * g.plane, false);
  if (inside) vc = src(col + (long long)z0 * g.plane, true);
  slab(sm, by, 0, ly + 1, lx + 1) = vc;
  fill_halo<T>(g, by, sm, 0, i0, j0, z0, src);
  __syncthreads();

  for (int k = z0; k < z1; k++) {
    const int buf = (k - z0) & 1;
    if (NDIM == 3) {
      vt = T(0);
      if (k + 1 < g.nz) {
        const bool own_next = (k + 1 < z1);
        if (inside) vt = src(col + (long long)(k + 1) * g.plane, own_next);
        if (own_next) {
          slab(sm, by, buf ^ 1, ly + 1, lx + 1) = vt;
          fill_halo<T>(g, by, sm, buf ^ 1, i0, j0, k + 1, src);
        }
      }
    }
    if (inside) {
      Nbr<T> nb;
      nb.c = vc;
      nb.w = slab(sm, by, buf, ly + 1, lx);
      nb.e = slab(sm, by, buf, ly + 1, lx + 2);
      nb.s = slab(sm, by, buf, ly, lx + 1);
      nb.n = slab(sm, by, buf, ly + 2, lx + 1);
      nb.b = vb;
      nb.t = vt;
      sink(col + (long long)k * g.plane, nb, i, j, k);
    }
    __syncthreads();
    vb = vc;
    vc = vt;
  }
}

// ---------------------------------------------------------------------------
// Stencil arithmetic.  Counts below are FP64-pipe instructions per node, the
// binding resource for FP64 on this GPU (2 lanes / clock / SM).
// ---------------------------------------------------------------------------

// Scaled operator, constant coefficients: returns (A x)_i / sigma where the
// host scaled all coefficients by 1/sigma so that the upper x coupling is
// exactly -1.  6 instructions in 3-D (4 in 2-D).
template <typename T, int OPK, int NDIM>
__device__ __forceinline__ T apply_unit(const Coef<T>& cf, const Nbr<T>& nb) {
  if (OPK == OP_SYM) {
    T y = fma(cf.d, nb.c, -(nb.w + nb.e));
    y = fma(cf.yl, nb.s + nb.n, y);
    if (NDIM == 3) y = fma(cf.zl, nb.b + nb.t, y);
    return y;
  } else {
    T y = fma(cf.d, nb.c, -nb.e);
    y = fma(cf.xl, nb.w, y);
    y = fma(cf.yl, nb.s, y);
    y = fma(cf.yu, nb.n, y);
    if (NDIM == 3) {
      y = fma(cf.zl, nb.b, y);
      y = fma(cf.zu, nb.t, y);
    }
    return y;
  }
}

// Variable-coefficient operator (sigma = 1): 7 instructions in 3-D.
template <typename T, int NDIM>
__device__ __forceinline__ T apply_vark(const Coef<T>& cf, const Geom& g, long long idx, int i, int j, int k,
                                        const Nbr<T>& nb) {
  T axu = (i + 1 < g.nx) ? __ldg(cf.ax + idx + 1) : T(0);
  T ayu = (j + 1 < g.ny) ? __ldg(cf.ay + idx + g.nx) : T(0);
  T y = __ldg(cf.D + idx) * nb.c;
  y = fma(-__ldg(cf.ax + idx), nb.w, y);
  y = fma(-axu, nb.e, y);
  y = fma(-__ldg(cf.ay + idx), nb.s, y);
  y = fma(-ayu, nb.n, y);
  if (NDIM == 3) {
    T azu = (k + 1 < g.nz) ? __ldg(cf.az + idx + g.plane) : T(0);
    y = fma(-__ldg(cf.az + idx), nb.b, y);
    y = fma(-azu, nb.t, y);
  }
  return y;
}

template <typename T, int OPK, int NDIM>
__device__ __forceinline__ T apply_op(const Coef<T>& cf, const Geom& g, long long idx, int i, int j, int k,
                                      const Nbr<T>& nb) {
  if (OPK == OP_VARK) return apply_vark<T, NDIM>(cf, g, idx, i, j, k, nb);
  return apply_unit<T, OPK, NDIM>(cf, nb);
}

// Jacobi update x' = (b - sum_{j!=i} a_ij x_j) / a_ii.  For constant
// coefficients the host passes g = -a/a_ii in the Coef slots and bD = b/a_ii
// (6 instructions in 3-D); for variable k, x' = (b + sum a x) * invD
// (7 instructions).  `bv` is bD (constant) or b (variable).
template <typename T, int OPK, int NDIM>
__device__ __forceinline__ T jacobi_update(const Coef<T>& cf, const Geom& g, long long idx, int i, int j, int k,
                                           const Nbr<T>& nb, T bv) {
  if (OPK == OP_SYM) {
    T y = fma(cf.xl, nb.w + nb.e, bv);
    y = fma(cf.yl, nb.s + nb.n, y);
    if (NDIM == 3) y = fma(cf.zl, nb.b + nb.t, y);
    return y;
  } else if (OPK == OP_NONSYM) {
    T y = fma(cf.xl, nb.w, bv);
    y = fma(cf.xu, nb.e, y);
    y = fma(cf.yl, nb.s, y);
    y = fma(cf.yu, nb.n, y);
    if (NDIM == 3) {
      y = fma(cf.zl, nb.b, y);
      y = fma(cf.zu, nb.t, y);
    }
    return y;
  } else {
    T axu = (i + 1 < g.nx) ? __ldg(cf.ax + idx + 1) : T(0);
    T ayu = (j + 1 < g.ny) ? __ldg(cf.ay + idx + g.nx) : T(0);
    T y = fma(__ldg(cf.ax + idx), nb.w, bv);
    y = fma(axu, nb.e, y);
    y = fma(__ldg(cf.ay + idx), nb.s, y);
    y = fma(ayu, nb.n, y);
    if (NDIM == 3) {
      T azu = (k + 1 < g.nz) ? __ldg(cf.az + idx + g.plane) : T(0);
      y = fma(__ldg(cf.az + idx), nb.b, y);
      y = fma(azu, nb.t, y);
    }
    return y * __ldg(cf.D + idx);  // D holds 1/a_ii for the Jacobi setup
  }
}

}  // namespace hs
