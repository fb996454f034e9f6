// hs_stencil.cuh -- the z-marching tile engine used by every stencil pass.
//
// A work item is an xy tile of (32 CX) x BY nodes (one warp per row, each
// lane owning CX columns 32 apart) and a range [z0, z1) of planes.  The block
// marches up the planes: each thread keeps the values of its own columns at
// planes k-1, k, k+1 in registers, while the plane k itself (tile plus a
// one-node halo) sits in a double-buffered shared-memory slab that supplies
// the W/E/S/N neighbours.  One __syncthreads per plane; with CX = 2 every
// thread carries two independent stencil chains per barrier.
//
// The stencil INPUT value at a node is produced by a functor `src` (a plain
// load for SpMV/Jacobi, or an on-the-fly vector update such as
// p = r + beta p for the Krylov passes); halo values are produced by whole
// warps (warp 0: row below, warp 1: row above, warp 2: the two side
// columns), so FP64 work is never issued for a handful of lanes.
// Nodes outside the grid read as zero (homogeneous Dirichlet ghosts).
#pragma once
#include <type_traits>

#include "hs_common.cuh"

namespace hs {

constexpr int BX = 32;

struct Tiling {
  int by;        // rows per tile (3..16), blockDim.x = 32 * by
  int tiles_x, tiles_y, chunks, lz;
  int cx;        // columns per lane (1 or 2): tile width 32 * cx
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
  i0 = tx * BX * t.cx;
  j0 = ty * t.by;
  z0 = c * t.lz;
  z1 = min(g.nz, z0 + t.lz);
}

// Shared slab: 2 planes of (by + 2) x (32 CX + 2) values.
template <typename T, int CX>
__device__ __forceinline__ T& slab(T* sm, int by, int buf, int row, int col) {
  return sm[(buf * (by + 2) + row) * (BX * CX + 2) + col];
}

// Neighbour values of the current node handed to the stencil functor (box:
// the sum over the node's 3x3x3 box, center included, for OP_BOX27 sinks).
template <typename T>
struct Nbr {
  T c, w, e, s, n, b, t;
  T box;
};

// A sink that applies the 27-point operator declares kBox = true; the tile
// engine then hands it box sums instead of the 7-point neighbourhood.
template <class S, class = void>
struct is_box_sink : std::false_type {};
template <class S>
struct is_box_sink<S, std::void_t<decltype(S::kBox)>> : std::integral_constant<bool, S::kBox> {};

// Process one work item, software-pipelined along z.
//
// The input functor `src` has two phases: src.fetch(idx) issues the loads
// of a node (returning a plain struct of raw values) and src.make(raw, idx,
// own) turns them into the stencil input (own = the node belongs to this
// item, so side outputs such as p may be stored).  The consumer `sink` has
// the same split: sink.fetch(idx, i, j, k) loads per-node operands (b, r',
// variable coefficients) and sink(idx, nb, raw, i, j, k) consumes the
// neighbourhood.  At plane step k the block issues the src loads of plane
// k+2 and the sink loads of plane k+1, then builds plane k+1 from loads
// issued one step earlier, then applies the stencil at plane k: global-memory
// latency is hidden behind a whole plane of work instead of sitting in front
// of the barrier.
//
// Halo nodes are produced by whole warps: warp 0 the row below the tile (CX
// nodes per lane), warp 1 the row above, warp 2 the two side columns (lanes
// 0..by-1 left, 16..16+by-1 right).  Requires 3 <= by <= 16 and tl.cx == CX.
template <typename T, class Src, class Sink>
__device__ __forceinline__ void zmarch_box(const Geom& g, const Tiling& tl, int item, T* sm, const Src& src,
                                           Sink& sink);

template <typename T, int NDIM, int CX, class Src, class Sink>
__device__ __forceinline__ void zmarch_item(const Geom& g, const Tiling& tl, int item, T* sm, const Src& src,
                                            Sink& sink) {
  if constexpr (is_box_sink<Sink>::value) {
    static_assert(NDIM == 3 && CX == 1, "the 27-point engine is 3-D with one column per lane");
    zmarch_box<T>(g, tl, item, sm, src, sink);
    return;
  }
  using SR = typename Src::Raw;
  using KR = typename Sink::Raw;
  constexpr int TW = BX * CX;
  int i0, j0, z0, z1;
  decode_item(tl, g, item, i0, j0, z0, z1);
  const int by = tl.by;
  const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
  const int j = j0 + ly;
  const long long P = g.plane;
  int ii[CX];
  bool inside[CX];
  long long col[CX];
#pragma unroll
  for (int c = 0; c < CX; c++) {
    ii[c] = i0 + lx + BX * c;
    inside[c] = (ii[c] < g.nx) && (j < g.ny);
    col[c] = (long long)j * g.nx + ii[c];
  }

  // halo nodes this thread produces (warps 0..2 only)
  constexpr int NH = CX;
  int hrow[NH], hcp[NH];
  bool hin[NH];
  long long hcol[NH];
#pragma unroll
  for (int c = 0; c < NH; c++) {
    hrow[c] = -1;
    hcp[c] = 0;
    hin[c] = false;
    hcol[c] = 0;
    int hi = 0, hj = 0;
    if (ly == 0) {
      hi = i0 + lx + BX * c; hj = j0 - 1; hrow[c] = 0; hcp[c] = lx + BX * c + 1;
    } else if (ly == 1) {
      hi = i0 + lx + BX * c; hj = j0 + by; hrow[c] = by + 1; hcp[c] = lx + BX * c + 1;
    } else if (ly == 2 && c == 0) {
      if (lx < by) {
        hi = i0 - 1; hj = j0 + lx; hrow[c] = lx + 1; hcp[c] = 0;
      } else if (lx >= 16 && lx < 16 + by) {
        hi = i0 + TW; hj = j0 + lx - 16; hrow[c] = lx - 15; hcp[c] = TW + 1;
      }
    }
    if (hrow[c] >= 0 && hi >= 0 && hi < g.nx && hj >= 0 && hj < g.ny) {
      hin[c] = true;
      hcol[c] = (long long)hj * g.nx + hi;
    }
  }

  T vb[CX], vc[CX], vt[CX];
  SR rown[CX], rhal[NH];   // raw src values of plane k+1
  KR kown[CX];             // raw sink values of plane k
#pragma unroll
  for (int c = 0; c < CX; c++) {
    vb[c] = T(0);
    vc[c] = T(0);
    vt[c] = T(0);
    rown[c] = SR{};
    rhal[c] = SR{};
    kown[c] = KR{};
  }
  {
    SR r0[CX], h0[NH];
#pragma unroll
    for (int c = 0; c < CX; c++) {
      r0[c] = SR{};
      h0[c] = SR{};
      if (NDIM == 3 && inside[c] && z0 > 0) {
        if (HS_IN_BOUNDS(col[c] + (long long)(z0 - 1) * P, g.N)) {
          SR rb = src.fetch(col[c] + (long long)(z0 - 1) * P);
          vb[c] = src.make(rb, col[c] + (long long)(z0 - 1) * P, false);
        }
      }
      if (inside[c] && HS_IN_BOUNDS(col[c] + (long long)z0 * P, g.N)) r0[c] = src.fetch(col[c] + (long long)z0 * P);
      if (hin[c] && HS_IN_BOUNDS(hcol[c] + (long long)z0 * P, g.N)) h0[c] = src.fetch(hcol[c] + (long long)z0 * P);
      if (inside[c] && HS_IN_BOUNDS(col[c] + (long long)z0 * P, g.N))
        kown[c] = sink.fetch(col[c] + (long long)z0 * P, ii[c], j, z0);
      if (NDIM == 3 && z0 + 1 < g.nz) {
        if (inside[c] && HS_IN_BOUNDS(col[c] + (long long)(z0 + 1) * P, g.N))
          rown[c] = src.fetch(col[c] + (long long)(z0 + 1) * P);
        if (hin[c] && z0 + 1 < z1 && HS_IN_BOUNDS(hcol[c] + (long long)(z0 + 1) * P, g.N))
          rhal[c] = src.fetch(hcol[c] + (long long)(z0 + 1) * P);
      }
    }
#pragma unroll
    for (int c = 0; c < CX; c++) {
      vc[c] = inside[c] ? src.make(r0[c], col[c] + (long long)z0 * P, true) : T(0);
      slab<T, CX>(sm, by, 0, ly + 1, lx + BX * c + 1) = vc[c];
      if (hrow[c] >= 0)
        slab<T, CX>(sm, by, 0, hrow[c], hcp[c]) = hin[c] ? src.make(h0[c], hcol[c] + (long long)z0 * P, false) : T(0);
    }
  }
  __syncthreads();

  for (int k = z0; k < z1; k++) {
    const int buf = (k - z0) & 1;
    SR rown2[CX], rhal2[NH];
    KR kown2[CX];
#pragma unroll
    for (int c = 0; c < CX; c++) {
      rown2[c] = SR{};
      rhal2[c] = SR{};
      kown2[c] = KR{};
    }
    if (NDIM == 3) {
#pragma unroll
      for (int c = 0; c < CX; c++) {
        if (inside[c] && k + 2 < g.nz && k + 2 <= z1 && HS_IN_BOUNDS(col[c] + (long long)(k + 2) * P, g.N))
          rown2[c] = src.fetch(col[c] + (long long)(k + 2) * P);
        if (hin[c] && k + 2 < z1 && HS_IN_BOUNDS(hcol[c] + (long long)(k + 2) * P, g.N))
          rhal2[c] = src.fetch(hcol[c] + (long long)(k + 2) * P);
        if (inside[c] && k + 1 < z1 && HS_IN_BOUNDS(col[c] + (long long)(k + 1) * P, g.N))
          kown2[c] = sink.fetch(col[c] + (long long)(k + 1) * P, ii[c], j, k + 1);
      }
#pragma unroll
      for (int c = 0; c < CX; c++) {
        vt[c] = T(0);
        if (k + 1 < g.nz) {
          const bool own_next = (k + 1 < z1);
          if (inside[c]) vt[c] = src.make(rown[c], col[c] + (long long)(k + 1) * P, own_next);
          if (own_next) {
            slab<T, CX>(sm, by, buf ^ 1, ly + 1, lx + BX * c + 1) = vt[c];
            if (hrow[c] >= 0)
              slab<T, CX>(sm, by, buf ^ 1, hrow[c], hcp[c]) =
                  hin[c] ? src.make(rhal[c], hcol[c] + (long long)(k + 1) * P, false) : T(0);
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < CX; c++) {
      if (inside[c]) {
        const int sx = lx + BX * c + 1;
        Nbr<T> nb;
        nb.c = vc[c];
        nb.w = slab<T, CX>(sm, by, buf, ly + 1, sx - 1);
        nb.e = slab<T, CX>(sm, by, buf, ly + 1, sx + 1);
        nb.s = slab<T, CX>(sm, by, buf, ly, sx);
        nb.n = slab<T, CX>(sm, by, buf, ly + 2, sx);
        nb.b = vb[c];
        nb.t = vt[c];
        if (HS_IN_BOUNDS(col[c] + (long long)k * P, g.N)) sink(col[c] + (long long)k * P, nb, kown[c], ii[c], j, k);
      }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < CX; c++) {
      vb[c] = vc[c];
      vc[c] = vt[c];
      rown[c] = rown2[c];
      rhal[c] = rhal2[c];
      kown[c] = kown2[c];
    }
  }
}

// The 27-point engine (OP_BOX27).  Same work items, source / sink functors
// and prefetch scheme as zmarch_item, one column per lane; the sink receives
// the node value c and its 3x3x3 box sum, formed separably so that a node
// costs 6 additions instead of 26:
//   Rx(i,j) = x(i-1,j) + x(i,j) + x(i+1,j)       rows j0-1 .. j0+by (shared)
//   P(i,j)  = Rx(i,j-1) + Rx(i,j) + Rx(i,j+1)     per column and plane
//   box_k   = P_k-1 + P_k + P_k+1                 per column, P kept in registers
// Plane k+1 is staged (tile plus a one-node ring including the corners),
// its row sums are formed, then its P, and the sink runs on plane k: two
// barriers per plane.  Halo producers: warp 0 the row below the tile, warp 1
// the row above, warp 2 the side columns, warp 3 lanes 0..3 the corners
// (requires 4 <= by <= 16).  Shared memory: the plane, (by + 2) x 34 values,
// then the row sums, (by + 2) x 32 values.
template <typename T, class Src, class Sink>
__device__ __forceinline__ void zmarch_box(const Geom& g, const Tiling& tl, int item, T* sm, const Src& src,
                                           Sink& sink) {
  using SR = typename Src::Raw;
  using KR = typename Sink::Raw;
  constexpr int SW = BX + 2;   // staged row width
  int i0, j0, z0, z1;
  decode_item(tl, g, item, i0, j0, z0, z1);
  const int by = tl.by;
  T* rx = sm + (by + 2) * SW;  // row sums, (by + 2) x BX
  const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
  const int i = i0 + lx, j = j0 + ly;
  const bool inside = (i < g.nx) && (j < g.ny);
  const long long P = g.plane;
  const long long col = (long long)j * g.nx + i;
  // the halo node of this thread (one at most)
  int hrow = -1, hcp = 0, hi = 0, hj = 0;
  if (ly == 0) {
    hi = i0 + lx; hj = j0 - 1; hrow = 0; hcp = lx + 1;
  } else if (ly == 1) {
    hi = i0 + lx; hj = j0 + by; hrow = by + 1; hcp = lx + 1;
  } else if (ly == 2) {
    if (lx < by) {
      hi = i0 - 1; hj = j0 + lx; hrow = lx + 1; hcp = 0;
    } else if (lx >= 16 && lx < 16 + by) {
      hi = i0 + BX; hj = j0 + lx - 16; hrow = lx - 15; hcp = BX + 1;
    }
  } else if (ly == 3 && lx < 4) {
    hi = (lx & 1) ? i0 + BX : i0 - 1;
    hj = (lx & 2) ? j0 + by : j0 - 1;
    hrow = (lx & 2) ? by + 1 : 0;
    hcp = (lx & 1) ? BX + 1 : 0;
  }
  const bool hin = hrow >= 0 && hi >= 0 && hi < g.nx && hj >= 0 && hj < g.ny;
  const long long hcol = hin ? (long long)hj * g.nx + hi : 0;

  // stage plane kk (values from raw loads issued earlier), form its row sums
  // and return P of this thread's column; planes outside the grid give 0
  auto plane_P = [&](int kk, const SR& rown, const SR& rhal, bool own, T& vown) -> T {
    vown = T(0);
    if (kk >= 0 && kk < g.nz) {
      if (inside) vown = src.make(rown, col + (long long)kk * P, own);
      sm[(ly + 1) * SW + lx + 1] = vown;
      if (hrow >= 0) sm[hrow * SW + hcp] = hin ? src.make(rhal, hcol + (long long)kk * P, false) : T(0);
    }
    __syncthreads();
    if (kk >= 0 && kk < g.nz) {
      const T* r = sm + (ly + 1) * SW + lx;
      rx[(ly + 1) * BX + lx] = (r[0] + r[1]) + r[2];
      if (ly < 2) {
        const int hr = ly == 0 ? 0 : by + 1;
        const T* q = sm + hr * SW + lx;
        rx[hr * BX + lx] = (q[0] + q[1]) + q[2];
      }
    }
    __syncthreads();
    if (kk < 0 || kk >= g.nz) return T(0);
    return (rx[ly * BX + lx] + rx[(ly + 1) * BX + lx]) + rx[(ly + 2) * BX + lx];
  };
  auto fetch_plane = [&](int kk, SR& rown, SR& rhal) {
    rown = SR{};
    rhal = SR{};
    if (kk >= 0 && kk < g.nz) {
      if (inside && HS_IN_BOUNDS(col + (long long)kk * P, g.N)) rown = src.fetch(col + (long long)kk * P);
      if (hin && HS_IN_BOUNDS(hcol + (long long)kk * P, g.N)) rhal = src.fetch(hcol + (long long)kk * P);
    }
  };

  // prologue: P of planes z0 - 1 and z0, the center value at z0
  SR ra, ha, rb, hb;
  fetch_plane(z0 - 1, ra, ha);
  fetch_plane(z0, rb, hb);
  T vdummy, vc;
  T Pm = plane_P(z0 - 1, ra, ha, false, vdummy);
  SR rn, hn;
  fetch_plane(z0 + 1, rn, hn);          // plane z0 + 1, staged in the first step
  KR kown = KR{};
  if (inside && HS_IN_BOUNDS(col + (long long)z0 * P, g.N)) kown = sink.fetch(col + (long long)z0 * P, i, j, z0);
  T Pc = plane_P(z0, rb, hb, true, vc);

  for (int k = z0; k < z1; k++) {
    // loads of the next step: src plane k + 2, sink operands of plane k + 1
    SR rn2, hn2;
    fetch_plane(k + 2 < z1 + 1 ? k + 2 : g.nz, rn2, hn2);
    KR kown2 = KR{};
    if (inside && k + 1 < z1 && HS_IN_BOUNDS(col + (long long)(k + 1) * P, g.N))
      kown2 = sink.fetch(col + (long long)(k + 1) * P, i, j, k + 1);
    T vt;
    const T Pn = plane_P(k + 1, rn, hn, k + 1 < z1, vt);
    if (inside) {
      Nbr<T> nb;
      nb.c = vc;
      nb.box = (Pm + Pc) + Pn;
      nb.w = nb.e = nb.s = nb.n = nb.b = nb.t = T(0);
      if (HS_IN_BOUNDS(col + (long long)k * P, g.N)) sink(col + (long long)k * P, nb, kown, i, j, k);
    }
    Pm = Pc;
    Pc = Pn;
    vc = vt;
    rn = rn2;
    hn = hn2;
    kown = kown2;
  }
  __syncthreads();   // the next item restages the shared plane
}

// Plain load of one vector as the stencil input.  CG = true reads through
// L2 only (data written earlier in the same persistent kernel).
template <typename T, bool CG>
struct LoadSrc {
  const T* x;
  struct Raw {
    T v;
  };
  __device__ __forceinline__ Raw fetch(long long idx) const { return Raw{CG ? __ldcg(x + idx) : __ldg(x + idx)}; }
  __device__ __forceinline__ T make(const Raw& r, long long, bool) const { return r.v; }
};

// ---------------------------------------------------------------------------
// Stencil arithmetic.  Counts below are FP64-pipe instructions per node, the
// binding resource for FP64 on this GPU (2 lanes / clock / SM).
// ---------------------------------------------------------------------------

// Per-node operator operands, prefetched one plane ahead.  Constant
// coefficients need none; variable coefficients carry the diagonal (or its
// inverse for the Jacobi form) and the six positive face couplings.
template <typename T, int OPK>
struct OpRaw {};
template <typename T>
struct OpRaw<T, OP_VARK> {
  T d, xl, xu, yl, yu, zl, zu;
};

template <typename T, int OPK, int NDIM>
__device__ __forceinline__ OpRaw<T, OPK> op_fetch(const Coef<T>& cf, const Geom& g, long long idx, int i, int j,
                                                  int k) {
  OpRaw<T, OPK> r{};
  if constexpr (OPK == OP_VARK) {
#ifdef HS_DEBUG
    if (!HS_IN_BOUNDS(idx, g.N) || (i + 1 < g.nx && !HS_IN_BOUNDS(idx + 1, g.N)) ||
        (j + 1 < g.ny && !HS_IN_BOUNDS(idx + g.nx, g.N)) || (NDIM == 3 && k + 1 < g.nz && !HS_IN_BOUNDS(idx + g.plane, g.N)))
      return r;
#endif
    r.d = __ldg(cf.D + idx);
    r.xl = __ldg(cf.ax + idx);
    r.xu = (i + 1 < g.nx) ? __ldg(cf.ax + idx + 1) : T(0);
    r.yl = __ldg(cf.ay + idx);
    r.yu = (j + 1 < g.ny) ? __ldg(cf.ay + idx + g.nx) : T(0);
    if (NDIM == 3) {
      r.zl = __ldg(cf.az + idx);
      r.zu = (k + 1 < g.nz) ? __ldg(cf.az + idx + g.plane) : T(0);
    }
  }
  return r;
}

// (A x)_i / sigma.  Constant coefficients: the host scaled every coupling by
// 1/sigma so that the upper x coupling is exactly -1 (6 FP64 instructions in
// 3-D, 4 in 2-D).  Variable coefficients (sigma = 1): 7 instructions.
template <typename T, int OPK, int NDIM>
__device__ __forceinline__ T op_apply(const Coef<T>& cf, const OpRaw<T, OPK>& o, const Nbr<T>& nb) {
  if constexpr (OPK == OP_BOX27) {
    // 27 c - (box - c), with cf.d = 28: 1 instruction after the box sums
    return fma(cf.d, nb.c, -nb.box);
  } else if constexpr (OPK == OP_SYM) {
    T y = fma(cf.d, nb.c, -(nb.w + nb.e));
    y = fma(cf.yl, nb.s + nb.n, y);
    if (NDIM == 3) y = fma(cf.zl, nb.b + nb.t, y);
    return y;
  } else if constexpr (OPK == OP_NONSYM) {
    T y = fma(cf.d, nb.c, -nb.e);
    y = fma(cf.xl, nb.w, y);
    y = fma(cf.yl, nb.s, y);
    y = fma(cf.yu, nb.n, y);
    if (NDIM == 3) {
      y = fma(cf.zl, nb.b, y);
      y = fma(cf.zu, nb.t, y);
    }
    return y;
  } else {
    T y = o.d * nb.c;
    y = fma(-o.xl, nb.w, y);
    y = fma(-o.xu, nb.e, y);
    y = fma(-o.yl, nb.s, y);
    y = fma(-o.yu, nb.n, y);
    if (NDIM == 3) {
      y = fma(-o.zl, nb.b, y);
      y = fma(-o.zu, nb.t, y);
    }
    return y;
  }
}

// Jacobi update x' = (b - sum_{j!=i} a_ij x_j) / a_ii.  Constant
// coefficients: the host passes g = -a/a_ii in the Coef slots and bv = b/a_ii
// (6 instructions in 3-D).  Variable coefficients: x' = (b + sum a x) * invD
// with o.d = 1/a_ii (7 instructions).
template <typename T, int OPK, int NDIM>
__device__ __forceinline__ T jacobi_apply(const Coef<T>& cf, const OpRaw<T, OPK>& o, const Nbr<T>& nb, T bv) {
  if constexpr (OPK == OP_BOX27) {
    // b/a_ii + (box - c)/27: the 26 neighbours all couple with -1
    return fma(cf.xl, nb.box - nb.c, bv);
  } else if constexpr (OPK == OP_SYM) {
    T y = fma(cf.xl, nb.w + nb.e, bv);
    y = fma(cf.yl, nb.s + nb.n, y);
    if (NDIM == 3) y = fma(cf.zl, nb.b + nb.t, y);
    return y;
  } else if constexpr (OPK == OP_NONSYM) {
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
    T y = fma(o.xl, nb.w, bv);
    y = fma(o.xu, nb.e, y);
    y = fma(o.yl, nb.s, y);
    y = fma(o.yu, nb.n, y);
    if (NDIM == 3) {
      y = fma(o.zl, nb.b, y);
      y = fma(o.zu, nb.t, y);
    }
    return y * o.d;
  }
}

}  // namespace hs
