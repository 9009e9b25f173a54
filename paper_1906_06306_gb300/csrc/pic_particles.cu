// Particle kernel of the PIC step: interp_em + push + comp_curr of Table 1
// (arXiv:1906.06306), one thread block per (tile, split).
//
// Particles are sorted by tile.  A block stages its tile's E and B plus a halo
// into shared memory, runs every particle of the tile's bucket (all species)
// through gather -> Boris -> move -> ZigZag and accumulates the current in a
// shared-memory window, which it finally adds into the global J planes.
//
// Shared-memory layout (x fastest inside each plane, wc = window cells):
//   1D: float4 (Ex, By, Bz, -) [half-staggered points], float4 (Ey, Ez, Bx, -)
//   2D: float2 (Ex, By) [(1/2,0)], float2 (Ey, Bx) [(0,1/2)], Ez [(0,0)], Bz [(1/2,1/2)]
//   3D: Ex Ey Ez Bx By Bz
//   then int32 Jx Jy Jz (fixed point) and float Jx Jy Jz (running sums).
// Components that share a stencil share their loads.  The current goes into
// the int32 window with native integer atomics (same-address lanes do not
// serialise) and is folded into the float window after every kSpillEvery
// batches of blockDim particles, before any int32 word can overflow.
//
// A particle whose stencil is not inside the window (it drifted more than
// halo-1 cells since the last sort) is a stray.  In 1D and 2D strays are put
// on a shared-memory queue and processed by the block, in full warps, through
// global memory, overlapped with the other blocks' work.  In 3D that global
// path would set the registers of the whole kernel (128 against 80: 2 against
// 3 resident blocks per SM), so strays are not touched: their warp appends
// them to the species' deferred list with one atomic, and k_particles_deferred
// runs them afterwards through global memory.  A move across the conducting
// wall is deferred the same way in every dimension.  Warps of in-window
// particles never diverge into a global path, and correctness never depends on
// the sort cadence.
#include <cmath>

#include "pic_kernels.h"

namespace pic {

// Window extents of a block: from the tuning at run time (FW0 = 0), or fixed
// at compile time for the common windows (FW0 x FW1 x FW2), which turns every
// shared-memory offset of the stencils and current words into a constant
// (measured 4.5 % faster on the 2D 16x8-tile window).  The launcher picks a
// fixed instantiation only when the tuning's window has exactly those extents.
template <int FW0, int FW1, int FW2>
struct Win {
  static __device__ __forceinline__ int w(const PushParams& P, int d) {
    if (FW0 > 0) return d == 0 ? FW0 : d == 1 ? FW1 : FW2;
    return P.t.W[d];
  }
  static __device__ __forceinline__ int wc(const PushParams& P) {
    return FW0 > 0 ? FW0 * FW1 * FW2 : P.t.wcells;
  }
  static __device__ __forceinline__ int ws(const PushParams& P) {
    return FW0 > 0 ? (FW0 * FW1 * FW2 + 3) / 4 * 4 : P.t.wstride;
  }
};

template <int D>
__host__ __device__ constexpr int field_floats() {
  return D == 1 ? 8 : (D == 2 && PIC_XPAIR) || (D == 3 && PIC_X3PAIR) ? 12 : 6;
}

// Words of the staged field region, rounded up so that the current planes
// that follow start on a 16-byte boundary (they are accessed as int4/float4).
__host__ __device__ inline int field_words(int nf, int wc) { return (nf * wc + 3) / 4 * 4; }

__device__ __forceinline__ float lerp(float a, float b, float w) { return fmaf(w, b - a, a); }

__device__ __forceinline__ float bilerp(float f00, float f10, float f01, float f11, float wx,
                                        float wy) {
  return lerp(lerp(f00, f10, wx), lerp(f01, f11, wx), wy);
}

// The same interpolation on two components at once with the packed FP32x2
// instructions of sm_100+ (one issue, two results): elementwise the very
// operations of lerp/bilerp, so the values are identical.
__device__ __forceinline__ float2 lerp2(float2 a, float2 b, float2 w) {
  return __ffma2_rn(w, __fadd2_rn(b, make_float2(-a.x, -a.y)), a);
}

__device__ __forceinline__ float2 bilerp2(float2 f00, float2 f10, float2 f01, float2 f11, float2 wx,
                                          float2 wy) {
  return lerp2(lerp2(f00, f10, wx), lerp2(f01, f11, wx), wy);
}

// Linear interpolation of one staggered 3D component (stag bit d: half a cell
// up axis d) from x-paired planes: FP[w] = (f(x), f(x+1)) at window cell w.
// The x lerps at the four (y, z) corners, then y, then z: interp1<3>'s order.
template <int STAG>
__device__ __forceinline__ float interp3x(const float2* FP, int W0, int W01, const int* l,
                                          const float* o) {
  int i0[3];
  float w[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (STAG & (1 << d)) {
      const bool up = o[d] >= 0.5f;
      i0[d] = up ? l[d] : l[d] - 1;
      w[d] = up ? o[d] - 0.5f : o[d] + 0.5f;
    } else {
      i0[d] = l[d];
      w[d] = o[d];
    }
  }
  const int i = i0[0] + W0 * i0[1] + W01 * i0[2];
  const float2 p00 = FP[i], p10 = FP[i + W0], p01 = FP[i + W01], p11 = FP[i + W0 + W01];
  const float a = lerp(p00.x, p00.y, w[0]), c = lerp(p10.x, p10.y, w[0]);
  const float a1 = lerp(p01.x, p01.y, w[0]), c1 = lerp(p11.x, p11.y, w[0]);
  const float r0 = lerp(a, c, w[1]), r1 = lerp(a1, c1, w[1]);
  return lerp(r0, r1, w[2]);
}

// Linear gather from the staged window (layout above), window-local cell l.
template <int D>
__device__ __forceinline__ void gather_smem(const float* sm, int wc, int W0, int W01, const int* l,
                                            const float* o, float* e, float* b) {
  if (D == 1) {
    const float4* FA = reinterpret_cast<const float4*>(sm);
    const float4* FB = reinterpret_cast<const float4*>(sm + 4 * wc);
    const bool hx = o[0] >= 0.5f;
    const int bh = hx ? l[0] : l[0] - 1;
    const float wh = hx ? o[0] - 0.5f : o[0] + 0.5f;
    const float4 a0 = FA[bh], a1 = FA[bh + 1];
    const float4 c0 = FB[l[0]], c1 = FB[l[0] + 1];
    e[0] = lerp(a0.x, a1.x, wh);
    b[1] = lerp(a0.y, a1.y, wh);
    b[2] = lerp(a0.z, a1.z, wh);
    e[1] = lerp(c0.x, c1.x, o[0]);
    e[2] = lerp(c0.y, c1.y, o[0]);
    b[0] = lerp(c0.z, c1.z, o[0]);
  } else if (D == 2 && PIC_XPAIR) {
    // x-paired layout: one 16-byte load per row for (Ex, By) and (Ey, Bx), one
    // 8-byte load per row for Ez and Bz; the same operations as below
    const float4* FA = reinterpret_cast<const float4*>(sm);
    const float4* FB = FA + wc;
    const float2* FC = reinterpret_cast<const float2*>(FB + wc);
    const float2* FD = FC + wc;
    const bool hx = o[0] >= 0.5f, hy = o[1] >= 0.5f;
    const int bxh = hx ? l[0] : l[0] - 1, byh = hy ? l[1] : l[1] - 1;
    const float wxh = hx ? o[0] - 0.5f : o[0] + 0.5f;
    const float wyh = hy ? o[1] - 0.5f : o[1] + 0.5f;
    int i = bxh + W0 * l[1];  // (1/2, 0): Ex, By
    const float4 a0 = FA[i], a1 = FA[i + W0];
    const float2 ra = bilerp2(make_float2(a0.x, a0.y), make_float2(a0.z, a0.w),
                              make_float2(a1.x, a1.y), make_float2(a1.z, a1.w),
                              make_float2(wxh, wxh), make_float2(o[1], o[1]));
    i = l[0] + W0 * byh;  // (0, 1/2): Ey, Bx
    const float4 b0 = FB[i], b1 = FB[i + W0];
    const float2 rb = bilerp2(make_float2(b0.x, b0.y), make_float2(b0.z, b0.w),
                              make_float2(b1.x, b1.y), make_float2(b1.z, b1.w),
                              make_float2(o[0], o[0]), make_float2(wyh, wyh));
    i = l[0] + W0 * l[1];  // (0, 0): Ez, paired with (1/2, 1/2): Bz
    const int k = bxh + W0 * byh;
    const float2 c0 = FC[i], c1 = FC[i + W0], d0 = FD[k], d1 = FD[k + W0];
    const float2 rc = bilerp2(make_float2(c0.x, d0.x), make_float2(c0.y, d0.y),
                              make_float2(c1.x, d1.x), make_float2(c1.y, d1.y),
                              make_float2(o[0], wxh), make_float2(o[1], wyh));
    e[0] = ra.x;
    b[1] = ra.y;
    e[1] = rb.x;
    b[0] = rb.y;
    e[2] = rc.x;
    b[2] = rc.y;
  } else if (D == 2) {
    const float2* FA = reinterpret_cast<const float2*>(sm);
    const float2* FB = reinterpret_cast<const float2*>(sm + 2 * wc);
    const float* FC = sm + 4 * wc;
    const float* FD = sm + 5 * wc;
    const bool hx = o[0] >= 0.5f, hy = o[1] >= 0.5f;
    const int bxh = hx ? l[0] : l[0] - 1, byh = hy ? l[1] : l[1] - 1;
    const float wxh = hx ? o[0] - 0.5f : o[0] + 0.5f;
    const float wyh = hy ? o[1] - 0.5f : o[1] + 0.5f;
    int i = bxh + W0 * l[1];  // (1/2, 0): Ex, By
    const float2 ra = bilerp2(FA[i], FA[i + 1], FA[i + W0], FA[i + W0 + 1],
                              make_float2(wxh, wxh), make_float2(o[1], o[1]));
    i = l[0] + W0 * byh;  // (0, 1/2): Ey, Bx
    const float2 rb = bilerp2(FB[i], FB[i + 1], FB[i + W0], FB[i + W0 + 1],
                              make_float2(o[0], o[0]), make_float2(wyh, wyh));
    i = l[0] + W0 * l[1];  // (0, 0): Ez, paired with (1/2, 1/2): Bz
    const int k = bxh + W0 * byh;
    const float2 rc = bilerp2(make_float2(FC[i], FD[k]), make_float2(FC[i + 1], FD[k + 1]),
                              make_float2(FC[i + W0], FD[k + W0]),
                              make_float2(FC[i + W0 + 1], FD[k + W0 + 1]),
                              make_float2(o[0], wxh), make_float2(o[1], wyh));
    e[0] = ra.x;
    b[1] = ra.y;
    e[1] = rb.x;
    b[0] = rb.y;
    e[2] = rc.x;
    b[2] = rc.y;
  } else if (PIC_X3PAIR) {
    // x-paired planes: one 8-byte load per (y, z) corner of a stencil, the
    // same operations in the same order as interp1<3>
    const float2* FP = reinterpret_cast<const float2*>(sm);
    e[0] = interp3x<1>(FP + EX * wc, W0, W01, l, o);
    e[1] = interp3x<2>(FP + EY * wc, W0, W01, l, o);
    e[2] = interp3x<4>(FP + EZ * wc, W0, W01, l, o);
    b[0] = interp3x<6>(FP + BX * wc, W0, W01, l, o);
    b[1] = interp3x<5>(FP + BY * wc, W0, W01, l, o);
    b[2] = interp3x<3>(FP + BZ * wc, W0, W01, l, o);
  } else {
    const SmemAcc A{const_cast<float*>(sm), W0, W01, wc};
    gather<3>(A, l, o, e, b);
  }
}

// Particle record as read from memory.
struct PRec {
  int cell;
  float o[3];
  float u[3];
};

template <int D, int MODE>
__device__ __forceinline__ void load_rec(const SpeciesDev& S, int p, PRec& r) {
  const long long n = S.ld;
  if (MODE == 2) {
    r.cell = S.cell_old[p];
#pragma unroll
    for (int d = 0; d < D; ++d) r.o[d] = S.off_old[d * n + p];
#pragma unroll
    for (int a = 0; a < 3; ++a) r.u[a] = S.u[a * n + p];
  } else {
    r.cell = S.rcell[p];
#pragma unroll
    for (int d = 0; d < D; ++d) r.o[d] = S.roff[d * n + p];
#pragma unroll
    for (int a = 0; a < 3; ++a) r.u[a] = S.ru[a * n + p];
  }
#pragma unroll
  for (int d = D; d < 3; ++d) r.o[d] = 0.f;
}

// First segment of a reflection at the conducting wall (the shock set-up of
// Sect. 4.2): the particle moved from the wall's cell (offsets o1) to below
// the wall plane (cell offset dc with dc[0] = -1, offsets o2; displacement
// dn).  Its current follows the true path: a straight segment to the point
// where it meets the wall plane, a fraction s = o1x / (o1x + 1 - o2x) of the
// move, then the mirrored remainder.  Writes the crossing point (cell offset
// e, offsets z) and the first segment's share w of dn on non-gridded axes.
template <int D>
__device__ __forceinline__ float wall_crossing(const int* dc, const float* o1, const float* o2,
                                               const float* dn, int* e, float* z, float* w) {
  const float s = o1[0] / (o1[0] + (1.0f - o2[0]));  // 1 - o2x is exact: o2x > 1/2
  e[0] = 0;
  z[0] = 0.f;
  w[0] = 0.f;
#pragma unroll
  for (int d = 1; d < 3; ++d) {
    if (d < D) {
      // crossing point relative to the old cell, kept between the two cells
      const float y = fmaf(s, (float)dc[d] + o2[d] - o1[d], o1[d]);
      const int lo = dc[d] < 0 ? dc[d] : 0, hi = dc[d] > 0 ? dc[d] : 0;
      int f = (int)floorf(y);
      f = f < lo ? lo : (f > hi ? hi : f);
      const float r = y - (float)f;
      e[d] = f;
      z[d] = r < 0.f ? 0.f : (r < 1.f ? r : 0.99999994f);
      w[d] = 0.f;
    } else {
      e[d] = 0;
      z[d] = 0.f;
      w[d] = s * dn[d];
    }
  }
  return s;
}

// What one_particle did with a particle.
enum : int { kDone = 0, kStray = 1, kWallCross = 2 };

// One particle through gather -> Boris -> move -> ZigZag.  PATH 0: the
// shared-memory window is used; a particle whose stencil leaves the window
// (kStray) is not touched.  PATH 1: everything goes through global memory
// (the 1D/2D in-block pass over the stray queue).  In both, a particle whose
// move crosses the conducting wall (kWallCross) is not touched either: the
// caller defers it.  PATH 2: global memory with the reflection applied here
// (the deferred and tail kernels).
//
// INTERIOR (PATH 0 only): the block's window lies inside the lattice on every
// axis, so window-local indices need no periodic wrap and a particle whose
// stencil is in the window moves to a cell inside the lattice: its new cell
// index is the old one plus the cell offsets times the axis strides.
template <int D, int MODE, int PATH, int FW0 = 0, int FW1 = 0, int FW2 = 1, bool INTERIOR = false,
          class JA = SmemJ>
__device__ __forceinline__ int one_particle(const PushParams& P, const SpeciesDev& S, int p,
                                            PRec r, const float* sm, const JA& SJ,
                                            const GlobAcc& GA, const int* w0, float qs) {
  constexpr bool GLOBAL = PATH != 0;
  const long long n = S.ld;
  // invalid data: cell outside the lattice, offset outside [0,1), non-finite u
  bool bad_off = false;
#pragma unroll
  for (int d = 0; d < D; ++d) bad_off |= !(r.o[d] >= 0.0f && r.o[d] < 1.0f);
  const bool bad_cell = (unsigned)r.cell >= (unsigned long long)P.g.plane;
  const bool bad_u = !(isfinite(r.u[0]) && isfinite(r.u[1]) && isfinite(r.u[2]));
  if (bad_cell | bad_off | bad_u) {
    atomicOr(P.status, (bad_cell ? ST_BAD_CELL : 0) | (bad_off ? ST_BAD_OFF : 0) |
                           (bad_u ? ST_BAD_U : 0));
    return kDone;
  }

  int ijk[3] = {0, 0, 0};
  {
    const int q = fdiv(r.cell, P.div0);
    ijk[0] = r.cell - q * P.g.n[0];
    if (D == 2) ijk[1] = q;  // q < n1: the cell is on the lattice
    if (D == 3) {
      ijk[2] = fdiv(q, P.div1);
      ijk[1] = q - ijk[2] * P.g.n[1];
    }
  }
  if (MODE == 3 && ijk[0] < P.wall) {  // behind the conducting wall
    atomicOr(P.status, ST_BEHIND_WALL);
    return kDone;
  }
  int l[3] = {0, 0, 0};
  if (!GLOBAL) {
    bool inwin = true;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      int v = ijk[d] - w0[d];
      if (!INTERIOR) {  // periodic image of the window
        if (P.wrap_fast) {
          v += (v < 0) ? P.g.n[d] : 0;
          v -= (v >= P.g.n[d]) ? P.g.n[d] : 0;
        } else {
          v = wrapi(v, P.g.n[d]);
        }
      }
      l[d] = v;
      inwin &= (unsigned)(v - 1) <= (unsigned)(Win<FW0, FW1, FW2>::w(P, d) - 4);
    }
    if (!inwin) return kStray;
  }

  float* u = r.u;
  const float* o1 = r.o;
  if (MODE != 2) {
    float e[3], b[3];
    if (GLOBAL)
      gather<D>(GA, ijk, o1, e, b);
    else
      gather_smem<D>(sm, Win<FW0, FW1, FW2>::wc(P), Win<FW0, FW1, FW2>::w(P, 0),
                     Win<FW0, FW1, FW2>::w(P, 0) * Win<FW0, FW1, FW2>::w(P, 1), l, o1, e, b);
    if (P.pusher == 1)
      higuera_cary(u, e, b, S.qm, P.g.c, P.inv_c, P.inv_c2);
    else
      boris(u, e, b, S.qm, P.g.c, P.inv_c, P.inv_c2);
  }
  float o2[3] = {0.f, 0.f, 0.f}, dn[3];
  int dc[3] = {0, 0, 0};
  move<D>(u, o1, P.g.c, o2, dc, dn);

  // A move that ends below the wall plane (only from the wall's own cell: a
  // step is shorter than one cell) is reflected: x -> 2 wall - x, u_x -> -u_x.
  // The tile kernel defers it (keeping the reflection out of the tile kernel
  // keeps its registers); the record is not written.
  const bool refl = MODE == 3 && ijk[0] + dc[0] < P.wall;
  if (PATH != 2 && refl) return kWallCross;

  if (MODE != 2) {
    int cell2;
    if (INTERIOR && !refl) {
      cell2 = r.cell + dc[0];
      if (D >= 2) cell2 += P.g.n[0] * dc[1];
      if (D == 3) cell2 += P.g.n[0] * P.g.n[1] * dc[2];
    } else {
      int nc[3] = {0, 0, 0};
#pragma unroll
      for (int d = 0; d < D; ++d) nc[d] = wrap1(ijk[d] + dc[d], P.g.n[d]);
      if (refl) nc[0] = ijk[0];
      cell2 = nc[0] + P.g.n[0] * (nc[1] + P.g.n[1] * nc[2]);
    }
    S.u[p] = refl ? -u[0] : u[0];
#pragma unroll
    for (int a = 1; a < 3; ++a) S.u[a * n + p] = u[a];
    S.off[p] = refl ? 1.0f - o2[0] : o2[0];
#pragma unroll
    for (int d = 1; d < D; ++d) S.off[d * n + p] = o2[d];
    S.cell[p] = cell2;
    if (MODE == 1) {
      S.cell_old[p] = r.cell;
#pragma unroll
      for (int d = 0; d < D; ++d) S.off_old[d * n + p] = o1[d];
    }
  }
  if (MODE != 1) {
    if (GLOBAL) {
      // one straight ZigZag move, or the two segments of a reflected one
      // (a single call site keeps the global pass small)
      int b[3] = {ijk[0], ijk[1], ijk[2]}, e[3] = {dc[0], dc[1], dc[2]};
      float a[3] = {o1[0], o1[1], o1[2]}, z[3] = {o2[0], o2[1], o2[2]};
      float w[3] = {dn[0], dn[1], dn[2]};
      if (refl) wall_crossing<D>(dc, o1, o2, dn, e, z, w);
#pragma unroll 1
      for (int seg = 0; seg < (refl ? 2 : 1); ++seg) {
        if (seg == 1) {
          // from the crossing point (cell b + e, offsets z) to the mirror
          // image of the end point (x offset 1 - o2x in the wall's cell)
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            b[d] = d < D ? wrap1(b[d] + e[d], P.g.n[d]) : 0;
            a[d] = z[d];
            w[d] = d < D ? 0.f : dn[d] - w[d];
            e[d] = d == 0 || d >= D ? 0 : dc[d] - e[d];
            z[d] = d == 0 ? 1.0f - o2[0] : o2[d];
          }
        }
        zigzag<D>(GA, b, e, a, z, w, S.q);
      }
    } else {
      zigzag<D>(SJ, l, dc, o1, o2, dn, qs);
    }
  }
  return kDone;
}

// TMA (1D/2D, modes 0 and 3, every record row 16-byte aligned): the records
// of each batch arrive in a shared-memory ring by bulk copies that thread 0
// issues one batch ahead (mbarriers `full` per stage, completed by the copies'
// bytes; `empty` per stage, one arrival per warp once it has read the stage).
// The batches start at the bucket's first index rounded down to a multiple of
// 4 (16-byte aligned copies); lanes outside [a, b) idle.
template <int D, int MODE, int FW0 = 0, int FW1 = 0, int FW2 = 1, bool TMA = false>
__global__ void __launch_bounds__(kPushThreads, D == 3 ? PIC_PUSH_MIN_BLOCKS_3D
                                                : TMA  ? PIC_PUSH_MIN_BLOCKS_TMA
                                                       : PIC_PUSH_MIN_BLOCKS)
    k_particles(const __grid_constant__ PushParams P) {
  extern __shared__ __align__(128) float sm[];
  static_assert(!TMA || D < 3, "the record stream is for the 1D/2D kernels");
  constexpr int NR = 1 + D + 3;  // record rows: cell, D offsets, 3 four-velocity components
  __shared__ unsigned long long bar_full[kRecStages], bar_empty[kRecStages];
  __shared__ int rng_a[kMaxSpecies], rng_b[kMaxSpecies];  // each species' particles [a, b)
  // 1D/2D: strays queued and processed by the block; 3D: deferred
  constexpr bool kDrain = D < 3;
  __shared__ int q_n;      // entries in the stray queue (1D/2D)
  __shared__ int n_stray;  // particles of this block deferred as strays (3D)
  const GlobAcc GA{P.F, P.g.plane, P.g.n[0], P.g.n[1], P.g.n[2]};
  const int tile = blockIdx.x / P.splits;
  const int split = blockIdx.x - tile * P.splits;
  const int tc[3] = {tile % P.t.nt[0], (tile / P.t.nt[0]) % P.t.nt[1],
                     tile / (P.t.nt[0] * P.t.nt[1])};
  int w0[3] = {0, 0, 0};
#pragma unroll
  for (int d = 0; d < D; ++d) w0[d] = tc[d] * P.t.T[d] - P.t.H;
  // the window lies inside the lattice: no periodic wrap (block-uniform)
  bool interior = PIC_INTERIOR != 0;
#pragma unroll
  for (int d = 0; d < D; ++d)
    interior &= w0[d] >= 0 && w0[d] + Win<FW0, FW1, FW2>::w(P, d) <= P.g.n[d];
  const int wc = Win<FW0, FW1, FW2>::wc(P);
  const int ws = Win<FW0, FW1, FW2>::ws(P);  // plane stride of the current windows (wc rounded up to 4)
  const int W0 = Win<FW0, FW1, FW2>::w(P, 0), W1 = Win<FW0, FW1, FW2>::w(P, 1);
  constexpr int NF = field_floats<D>();
  const int fw = field_words(NF, wc);
  // fixed-point window: 3 planes of int32 words, or (2D, kJ64<D>) of 64-bit
  // pairs of them; then the float running sums and the 1D/2D stray queue
  constexpr int JW = kJ64<D> ? 6 : 3;  // words per window cell of the int window
  // float running sums of the current (none where folds go to global memory)
  constexpr int JF = kFoldGlobal<D> ? 0 : 3;
  int* ji = reinterpret_cast<int*>(sm + fw);
  float* jf = sm + fw + JW * ws;
  int* queue = reinterpret_cast<int*>(sm + fw + (JW + JF) * ws);  // kDrain only
  using JAcc = typename std::conditional<kJ64<D>, SmemJ64, SmemJ>::type;
  JAcc SJ;
  if constexpr (kJ64<D>)
    SJ = SmemJ64{reinterpret_cast<unsigned long long*>(ji), W0, ws};
  else
    SJ = SmemJ{ji, W0, W0 * W1, ws};
  const int lane = threadIdx.x & 31;

  float* ring = reinterpret_cast<float*>(queue + kQueueCap);  // TMA only
  // the particles of this block: a contiguous share of each species' tile bucket
  auto bucket = [&](int s, int& a, int& b) {
    const SpeciesDev& S = P.sp[s];
    const long long lo = S.tstart[tile * P.t.nsub], hi = S.tstart[(tile + 1) * P.t.nsub];
    const long long len = hi - lo;
    a = (int)(lo + len * split / P.splits);
    b = (int)(lo + len * (split + 1) / P.splits);
  };
  // producer state of the record stream (thread 0): species and first index of
  // the next batch to issue; pr_s == nspecies when everything is issued
  // (in shared memory: only thread 0 uses it, and registers are scarce)
  __shared__ struct {
    int s, base;  // species and first index of the next batch to issue (s == nspecies: done)
    int issued;   // batches issued
    int seen;     // batches thread 0 found complete
  } pr;
  auto pr_next_species = [&](int s) {
    while (s < P.nspecies && rng_a[s] >= rng_b[s]) ++s;
    pr.s = s;
    if (s < P.nspecies) pr.base = rng_a[s] & ~3;
  };
  // issue batch j (the producer's next) into stage j % kRecStages
  auto pr_issue = [&](int j) {
    const SpeciesDev& S = P.sp[pr.s];
    const int base = pr.base;
    const int end4 = (rng_b[pr.s] + 3) & ~3;
    const int cnt = end4 - base < kPushThreads ? end4 - base : kPushThreads;
    const unsigned bytes = 4u * (unsigned)cnt;
    unsigned long long* bar = &bar_full[j % kRecStages];
    float* dst = ring + (j % kRecStages) * NR * kPushThreads;
    mbar_arrive_expect_tx(bar, bytes * NR);
    bulk_load(dst, S.rcell + base, bytes, bar);
#pragma unroll
    for (int d = 0; d < D; ++d) bulk_load(dst + (1 + d) * kPushThreads, S.roff + d * S.ld + base, bytes, bar);
#pragma unroll
    for (int a = 0; a < 3; ++a)
      bulk_load(dst + (1 + D + a) * kPushThreads, S.ru + a * S.ld + base, bytes, bar);
    pr.issued = j + 1;
    pr.base = base + kPushThreads;
    if (pr.base >= rng_b[pr.s]) pr_next_species(pr.s + 1);
  };
  bool dead = false;  // this thread gave up on the stream after a timed-out wait

  if (threadIdx.x == 0) {
    q_n = 0;
    n_stray = 0;
    if (TMA) {
      for (int s = 0; s < P.nspecies; ++s) bucket(s, rng_a[s], rng_b[s]);
      for (int k = 0; k < kRecStages; ++k) {
        mbar_init(&bar_full[k], 1);
        mbar_init(&bar_empty[k], blockDim.x / 32);
      }
      mbar_init_fence();
      pr.issued = 0;
      pr.seen = 0;
      pr_next_species(0);
      if (pr.s < P.nspecies) pr_issue(0);  // overlaps the window staging
    }
  }
  // 2D, window inside the lattice: E and B of the window (with its guard
  // cells) arrive by one tensor copy into the current and queue area, which is
  // not in use yet; the loop below reads them there instead of global memory
  __shared__ unsigned long long bar_win;
  const bool win_tma = D == 2 && MODE != 2 && !TMA && P.win_tma != 0 && interior;
  // tensor copies land on a 128-byte boundary (at most 31 floats of padding)
  const float* land =
      reinterpret_cast<const float*>((reinterpret_cast<uintptr_t>(sm + fw) + 127) & ~uintptr_t(127));
  if (win_tma) {
    if (threadIdx.x == 0) {
      mbar_init(&bar_win, 1);
      mbar_init_fence();
      mbar_arrive_expect_tx(&bar_win, 24u * (unsigned)(P.win_box[0] * P.win_box[1]));
      tensor_load_3d(const_cast<float*>(land), &P.win_map, w0[0] - P.win_shift, w0[1], 0,
                     &bar_win);
    }
    __syncthreads();  // the barrier is initialised before anyone waits on it
    const bool landed = mbar_wait(&bar_win, 0, P.status);
    // a copy that did not land in time (the status word says so): the block
    // leaves, all of it, once a second bounded wait has seen the copy land or
    // expired too
    if (__syncthreads_or(!landed)) {
      if (threadIdx.x == 0) mbar_wait(&bar_win, 0, nullptr);
      return;
    }
  }
  for (int w = threadIdx.x; w < wc; w += blockDim.x) {
    const int lx = w % W0, rr = w / W0, ly = rr % W1, lz = rr / W1;
    const long long gi = GA.at(w0[0] + lx, w0[1] + ly, w0[2] + lz);
    if (MODE != 2) {
      float ex, ey, ez, bx, by, bz;
      if (win_tma) {  // box planes Ex .. Bz of box_x x box_y floats, x fastest
        const int pl = P.win_box[0] * P.win_box[1];
        const float* L = land + ly * P.win_box[0] + lx + P.win_shift;
        ex = L[0];
        ey = L[pl];
        ez = L[2 * pl];
        bx = L[3 * pl];
        by = L[4 * pl];
        bz = L[5 * pl];
      } else {
        ex = __ldg(&P.F[EX * P.g.plane + gi]);
        ey = __ldg(&P.F[EY * P.g.plane + gi]);
        ez = __ldg(&P.F[EZ * P.g.plane + gi]);
        bx = __ldg(&P.F[BX * P.g.plane + gi]);
        by = __ldg(&P.F[BY * P.g.plane + gi]);
        bz = __ldg(&P.F[BZ * P.g.plane + gi]);
      }
      if (D == 1) {
        reinterpret_cast<float4*>(sm)[w] = make_float4(ex, by, bz, 0.f);
        reinterpret_cast<float4*>(sm + 4 * wc)[w] = make_float4(ey, ez, bx, 0.f);
      } else if (D == 2 && PIC_XPAIR) {
        // point x goes to the low half of its own cell's pair and to the high
        // half of the pair of the cell before it (the last column's high half
        // is never read: stencils end at W0 - 2)
        float4* FA = reinterpret_cast<float4*>(sm);
        float4* FB = FA + wc;
        float2* FC = reinterpret_cast<float2*>(FB + wc);
        float2* FD = FC + wc;
        reinterpret_cast<float2*>(FA + w)[0] = make_float2(ex, by);
        reinterpret_cast<float2*>(FB + w)[0] = make_float2(ey, bx);
        FC[w].x = ez;
        FD[w].x = bz;
        if (lx > 0) {
          reinterpret_cast<float2*>(FA + w - 1)[1] = make_float2(ex, by);
          reinterpret_cast<float2*>(FB + w - 1)[1] = make_float2(ey, bx);
          FC[w - 1].y = ez;
          FD[w - 1].y = bz;
        }
      } else if (D == 2) {
        reinterpret_cast<float2*>(sm)[w] = make_float2(ex, by);
        reinterpret_cast<float2*>(sm + 2 * wc)[w] = make_float2(ey, bx);
        sm[4 * wc + w] = ez;
        sm[5 * wc + w] = bz;
      } else if (PIC_X3PAIR) {
        // point x goes to the low half of its own cell's pair and to the high
        // half of the pair of the cell before it (the last column's high half
        // is never read: stencils end at W0 - 2)
        float2* FP = reinterpret_cast<float2*>(sm);
        const float v[6] = {ex, ey, ez, bx, by, bz};
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          FP[c * wc + w].x = v[c];
          if (lx > 0) FP[c * wc + w - 1].y = v[c];
        }
      } else {
        sm[EX * wc + w] = ex;
        sm[EY * wc + w] = ey;
        sm[EZ * wc + w] = ez;
        sm[BX * wc + w] = bx;
        sm[BY * wc + w] = by;
        sm[BZ * wc + w] = bz;
      }
    }
  }
  if (win_tma) __syncthreads();  // the landing area is read before it is cleared
  if (MODE != 1) {
    int4* j4 = reinterpret_cast<int4*>(ji);
    for (int w = threadIdx.x; w < (JW + JF) * ws / 4; w += blockDim.x)
      j4[w] = make_int4(0, 0, 0, 0);
  }
  __syncthreads();

  // between barriers: fold the int32 window into the float window, clear it
  auto spill = [&]() {
    if constexpr (kFoldGlobal<D>) {
      // the fixed-point sums go straight to the global J planes, then are cleared
      for (int c = 0; c < 3; ++c) {
        for (int w = threadIdx.x; w < wc; w += blockDim.x) {
          const int v = ji[c * ws + w];
          if (v != 0) {
            const int lx = w % W0, rr = w / W0, ly = rr % W1, lz = rr / W1;
            const long long gi = GA.at(w0[0] + lx, w0[1] + ly, w0[2] + lz);
            atomicAdd(&P.F[(JX + c) * P.g.plane + gi], (float)v * P.jq);
            ji[c * ws + w] = 0;
          }
        }
      }
      return;
    }
    if constexpr (kJ64<D>) {
      // every float word gathers its two partial sums (SmemJ64's planes),
      // then, after all threads have read, the pairs are cleared
      const unsigned long long* Q = reinterpret_cast<const unsigned long long*>(ji);
      const unsigned long long* R = Q + ws;
      const unsigned long long* Pz = Q + 2 * ws;
      for (int w = threadIdx.x; w < wc; w += blockDim.x) {
        const bool x0 = w % W0 == 0, y0 = w < W0;
        const unsigned long long q = Q[w], p = Pz[w];
        const unsigned long long ry = y0 ? 0ULL : R[w - W0], rx = x0 ? 0ULL : R[w - 1];
        const unsigned long long px = x0 ? 0ULL : Pz[w - 1];
        const int vx = SmemJ64::lo(q) + SmemJ64::lo(ry);
        const int vy = SmemJ64::hi(q) + SmemJ64::hi(rx);
        const int vz = SmemJ64::lo(p) + SmemJ64::hi(px);
        if (vx != 0) jf[w] = fmaf((float)vx, P.jq, jf[w]);
        if (vy != 0) jf[ws + w] = fmaf((float)vy, P.jq, jf[ws + w]);
        if (vz != 0) jf[2 * ws + w] = fmaf((float)vz, P.jq, jf[2 * ws + w]);
      }
      __syncthreads();
      int4* i4 = reinterpret_cast<int4*>(ji);
      for (int w = threadIdx.x; w < 6 * ws / 4; w += blockDim.x) i4[w] = make_int4(0, 0, 0, 0);
      return;
    }
    int4* i4 = reinterpret_cast<int4*>(ji);
    float4* f4 = reinterpret_cast<float4*>(jf);
    for (int w = threadIdx.x; w < 3 * ws / 4; w += blockDim.x) {
      const int4 v = i4[w];
      if ((v.x | v.y | v.z | v.w) != 0) {
        float4 f = f4[w];
        f.x = fmaf((float)v.x, P.jq, f.x);
        f.y = fmaf((float)v.y, P.jq, f.y);
        f.z = fmaf((float)v.z, P.jq, f.z);
        f.w = fmaf((float)v.w, P.jq, f.w);
        f4[w] = f;
        i4[w] = make_int4(0, 0, 0, 0);
      }
    }
  };
  // 1D/2D: process the queued strays through global memory, then empty the
  // queue (a wall crosser among them is deferred)
  auto drain = [&](const SpeciesDev& S, int cnt) {
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      PRec r;
      load_rec<D, MODE>(S, queue[i], r);
      if (one_particle<D, MODE, 1, FW0, FW1, FW2>(P, S, queue[i], r, sm, SJ, GA, w0, 0.f) ==
          kWallCross)
        S.dlist[atomicAdd(S.dcount, 1)] = queue[i];
    }
    if (threadIdx.x == 0) atomicAdd(P.strays, (unsigned long long)cnt);
    __syncthreads();
    if (threadIdx.x == 0) q_n = 0;
    __syncthreads();
  };

  // Particles kPushThreads at a time (with PIC_PREFETCH the record of the next
  // batch is loaded while the current one is processed).  Every kSpillEvery
  // batches (and only there) the block synchronises, folds the current and, in
  // 1D/2D, drains the stray queue if it could overflow in the next round.
  int batches = 0;
  int kk = 0;  // batches of every species so far (the record stream's index)
  for (int s = 0; s < P.nspecies; ++s) {
    const SpeciesDev& S = P.sp[s];
    int a, b;
    if (TMA) {
      a = rng_a[s];
      b = rng_b[s];
    } else {
      bucket(s, a, b);
    }
    const float qs = S.q * P.jq_inv;
    PRec cur, nxt;
    if (PIC_PREFETCH && !TMA && a + (int)threadIdx.x < b) load_rec<D, MODE>(S, a + threadIdx.x, cur);
    // block-uniform trip count; with the stream the batches start 16-byte aligned
    for (int base = TMA && a < b ? a & ~3 : a; base < b; base += blockDim.x) {
      const int p = base + threadIdx.x;
      bool in = p >= a && p < b;
      if (TMA) {
        const int stage = kk % kRecStages;
        if (!dead) {
          if (!mbar_wait(&bar_full[stage], (kk / kRecStages) & 1, P.status))
            dead = true;
          else if (threadIdx.x == 0)
            pr.seen = kk + 1;
        }
        if (in && !dead) {
          const float* rec = ring + stage * NR * kPushThreads + threadIdx.x;
          cur.cell = __float_as_int(rec[0]);
#pragma unroll
          for (int d = 0; d < D; ++d) cur.o[d] = rec[(1 + d) * kPushThreads];
#pragma unroll
          for (int d = D; d < 3; ++d) cur.o[d] = 0.f;
#pragma unroll
          for (int c = 0; c < 3; ++c) cur.u[c] = rec[(1 + D + c) * kPushThreads];
        }
        in &= !dead;
        __syncwarp();
        if (lane == 0) mbar_arrive(&bar_empty[stage]);
        if (threadIdx.x == 0 && pr.s < P.nspecies && !dead) {
          // batch j = kk + 1 reuses the stage that batch j - kRecStages read
          const int j = pr.issued;
          if (j < kRecStages ||
              mbar_wait(&bar_empty[j % kRecStages], ((j - kRecStages) / kRecStages) & 1, P.status))
            pr_issue(j);
          else
            dead = true;
        }
        ++kk;
      } else if (PIC_PREFETCH) {
        if (p + (int)blockDim.x < b) load_rec<D, MODE>(S, p + blockDim.x, nxt);
      } else if (in) {
        load_rec<D, MODE>(S, p, cur);
      }
      int st = kDone;
      if (in)
        st = interior ? one_particle<D, MODE, 0, FW0, FW1, FW2, true>(P, S, p, cur, sm, SJ, GA, w0, qs)
                      : one_particle<D, MODE, 0, FW0, FW1, FW2>(P, S, p, cur, sm, SJ, GA, w0, qs);
      if (kDrain && st == kStray) {
        const int slot = atomicAdd(&q_n, 1);
        if (slot < kQueueCap) {
          queue[slot] = p;
        } else {  // full queue: this lane runs the stray through global memory now
          if (one_particle<D, MODE, 1, FW0, FW1, FW2>(P, S, p, cur, sm, SJ, GA, w0, 0.f) ==
              kWallCross)
            S.dlist[atomicAdd(S.dcount, 1)] = p;
          atomicAdd(P.strays, 1ULL);
        }
      }
      if (!kDrain || MODE == 3) {
        // deferred particles: one list slot range per warp, reserved by one atomic
        const bool dfr = kDrain ? st == kWallCross : st != kDone;
        const unsigned defer = __ballot_sync(0xffffffffu, dfr);
        if (defer) {
          const unsigned strays = __ballot_sync(0xffffffffu, st == kStray);
          const int leader = __ffs(defer) - 1;
          int at = 0;
          if (lane == leader) {
            at = atomicAdd(S.dcount, __popc(defer));
            if (!kDrain && strays) atomicAdd(&n_stray, __popc(strays));
          }
          at = __shfl_sync(0xffffffffu, at, leader);
          if (dfr) S.dlist[at + __popc(defer & lanemask_lt())] = p;
        }
      }
      if (PIC_PREFETCH) cur = nxt;
      if (++batches == kSpillEvery) {
        batches = 0;
        __syncthreads();
        const int qn = q_n;  // read by every thread before anyone can queue again
        if (MODE != 1) spill();
        __syncthreads();
        if (kDrain && qn > kQueueCap / 2) drain(S, qn < kQueueCap ? qn : kQueueCap);
      }
    }
    if (kDrain) {  // end of species: everything queued for it is processed before the next
      __syncthreads();
      const int qn = q_n;
      __syncthreads();
      if (qn > 0) drain(S, qn < kQueueCap ? qn : kQueueCap);
    }
  }

  if (TMA && threadIdx.x == 0) {
    // after a timed-out wait: copies issued but never found complete must land
    // before the block's shared memory is released
    for (int j = pr.seen; j < pr.issued; ++j)
      mbar_wait(&bar_full[j % kRecStages], (j / kRecStages) & 1, nullptr);
  }
  __syncthreads();
  if (threadIdx.x == 0 && n_stray > 0) atomicAdd(P.strays, (unsigned long long)n_stray);
  if (MODE != 1) {
    spill();
    __syncthreads();
    for (int w = threadIdx.x; w < (kFoldGlobal<D> ? 0 : wc); w += blockDim.x) {
      const int lx = w % W0, rr = w / W0, ly = rr % W1, lz = rr / W1;
      const long long gi = GA.at(w0[0] + lx, w0[1] + ly, w0[2] + lz);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float v = jf[c * ws + w];
        if (v != 0.0f) atomicAdd(&P.F[(JX + c) * P.g.plane + gi], v);
      }
    }
  }
}

// Particles appended (injected) since the last sort belong to no tile bucket
// yet: they take the global-memory path, grid-strided over [tail, n).
template <int D>
__global__ void __launch_bounds__(kPushThreads) k_particles_tail(const PushParams P) {
  const GlobAcc GA{P.F, P.g.plane, P.g.n[0], P.g.n[1], P.g.n[2]};
  for (int s = 0; s < P.nspecies; ++s) {
    const SpeciesDev& S = P.sp[s];
    for (long long p = S.tail + (long long)blockIdx.x * blockDim.x + threadIdx.x; p < S.n;
         p += (long long)gridDim.x * blockDim.x) {
      PRec r;
      load_rec<D, 3>(S, (int)p, r);
      one_particle<D, 3, 2>(P, S, (int)p, r, nullptr, SmemJ{nullptr, 0, 0, 0}, GA, nullptr, 0.f);
    }
  }
}

// Particles that k_particles deferred (strays outside their tile window, and
// moves across the conducting wall): the whole update through global memory,
// with the reflection.  Their records were not written, so they are read
// where k_particles read them; each slot is listed at most once per launch.
template <int D, int MODE>
__global__ void __launch_bounds__(kPushThreads) k_particles_deferred(const PushParams P) {
  const GlobAcc GA{P.F, P.g.plane, P.g.n[0], P.g.n[1], P.g.n[2]};
  for (int s = 0; s < P.nspecies; ++s) {
    const SpeciesDev& S = P.sp[s];
    const int cnt = *S.dcount;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
      const int p = S.dlist[i];
      PRec r;
      load_rec<D, MODE>(S, p, r);
      one_particle<D, MODE, 2>(P, S, p, r, nullptr, SmemJ{nullptr, 0, 0, 0}, GA, nullptr, 0.f);
    }
  }
}

long long window_landing_floats(int dim, const TileDev& t) {
  const int nf = dim == 1 ? field_floats<1>() : dim == 2 ? field_floats<2>() : field_floats<3>();
  // the landing area starts on the first 128-byte boundary past the field words
  return (long long)(particle_smem_bytes(dim, t) / sizeof(float)) - field_words(nf, t.wcells) - 31;
}

size_t particle_smem_bytes(int dim, const TileDev& t) {
  const int nf = dim == 1 ? field_floats<1>() : dim == 2 ? field_floats<2>() : field_floats<3>();
  const int jw = (dim == 2 && kJ64<2>) ? 6 : 3;  // int window words per cell
  const int jf = dim == 3 && kFoldGlobal<3> ? 0 : 3;  // float window words per cell
  // 1D/2D: the stray queue and the ring of streamed particle records
  const size_t ring = PIC_TMA_RECORDS ? (size_t)kRecStages * (1 + dim + 3) * kPushThreads : 0;
  size_t words = (size_t)(jw + jf) * t.wstride + (dim < 3 ? kQueueCap + ring : 0);
  // 2D: the same area first takes the window's tensor copy, E and B over a box
  // whose x extent is the window's widened to 16-byte ends, after up to 31
  // floats of padding to a 128-byte boundary
  if (dim == 2 && PIC_TMA_WINDOW) {
    const int shift = ((-t.H) % 4 + 4) % 4;
    const size_t box = 6 * (size_t)((t.W[0] + shift + 3) / 4 * 4) * t.W[1] + 31;
    words = box > words ? box : words;
  }
  return sizeof(float) * ((size_t)field_words(nf, t.wcells) + words);
}

float current_quantum(float max_abs_q, float c, int batch) {
  const double bound = 1.25 * (double)c * (double)batch * (double)max_abs_q;
  const int e = (int)std::ceil(std::log2(bound > 0 ? bound : 1.0));
  return (float)std::ldexp(1.0, e - 31);
}

FastDiv make_fastdiv(int d) {
  int l = 0;
  while ((1LL << l) < (long long)d) ++l;  // ceil(log2 d)
  const int s = 31 + l;
  const unsigned long long two_s = 1ULL << s;
  FastDiv f;
  f.M = (two_s + (unsigned long long)d - 1) / (unsigned long long)d;
  f.s = s;
  f.d = d;
  return f;
}

template <int D, int MODE, int FW0 = 0, int FW1 = 0, int FW2 = 1, bool TMA = false>
static cudaError_t set_limit(int bytes) {
  return cudaFuncSetAttribute(k_particles<D, MODE, FW0, FW1, FW2, TMA>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t set_particle_smem_limit(int bytes) {
  cudaError_t e = cudaSuccess;
#define PIC_SET(D)                                  \
  if (e == cudaSuccess) e = set_limit<D, 0>(bytes); \
  if (e == cudaSuccess) e = set_limit<D, 1>(bytes); \
  if (e == cudaSuccess) e = set_limit<D, 2>(bytes); \
  if (e == cudaSuccess) e = set_limit<D, 3>(bytes);
  PIC_SET(1)
  PIC_SET(2)
  PIC_SET(3)
#undef PIC_SET
  if (e == cudaSuccess) e = set_limit<2, 0, 23, 15>(bytes);
  if (e == cudaSuccess) e = set_limit<2, 0, 23, 23>(bytes);
  if (e == cudaSuccess) e = set_limit<2, 0, 25, 17>(bytes);
#if PIC_TMA_RECORDS
  if (e == cudaSuccess) e = set_limit<2, 0, 23, 15, 1, true>(bytes);
  if (e == cudaSuccess) e = set_limit<2, 0, 23, 23, 1, true>(bytes);
  if (e == cudaSuccess) e = set_limit<1, 0, 0, 0, 1, true>(bytes);
  if (e == cudaSuccess) e = set_limit<1, 3, 0, 0, 1, true>(bytes);
  if (e == cudaSuccess) e = set_limit<2, 0, 0, 0, 1, true>(bytes);
  if (e == cudaSuccess) e = set_limit<2, 3, 0, 0, 1, true>(bytes);
#endif
  if (e == cudaSuccess) e = set_limit<3, 0, 13, 13, 9>(bytes);
  if (e == cudaSuccess) e = set_limit<3, 3, 13, 13, 9>(bytes);
  if (e == cudaSuccess) e = set_limit<3, 0, 13, 13, 7>(bytes);
  if (e == cudaSuccess) e = set_limit<3, 3, 13, 13, 7>(bytes);
  return e;
}

template <int D, int MODE>
static cudaError_t launch(const PushParams& P, cudaStream_t st) {
  const unsigned nblocks = (unsigned)P.t.ntiles * (unsigned)P.splits;
  // the deferred lists can have entries in 3D (strays) and with the wall
  constexpr bool deferred = D == 3 || MODE == 3;
  if (deferred) {
    const cudaError_t e = cudaMemsetAsync(P.dcount, 0, sizeof(int) * P.nspecies, st);
    if (e != cudaSuccess) return e;
  }
  const size_t smem = particle_smem_bytes(D, P.t);
  // fixed-window instantiations: 2D windows of 16x8 and 16x16 tiles with
  // halo 3 (23 x 15, 23 x 23) and of 16x8 tiles with halo 4 (25 x 17), the 3D
  // window of 8x8x4 tiles with halo 2 (13 x 13 x 9); any other window takes
  // the generic kernel
  const bool w3 = P.t.W[0] == 13 && P.t.W[1] == 13 && P.t.W[2] == 9;
  const bool w37 = P.t.W[0] == 13 && P.t.W[1] == 13 && P.t.W[2] == 7;  // 8x8x2 tiles, halo 2
  // the record stream needs 16-byte aligned rows (bulk copies)
  constexpr bool kStreamable = PIC_TMA_RECORDS && D < 3 && (MODE == 0 || MODE == 3);
  const bool tma = kStreamable && P.rec_aligned;
  if (D == 2 && MODE == 0 && P.t.W[0] == 23 && P.t.W[1] == 15 && tma)
    k_particles<2, 0, 23, 15, 1, kStreamable><<<nblocks, kPushThreads, smem, st>>>(P);
  else if (D == 2 && MODE == 0 && P.t.W[0] == 23 && P.t.W[1] == 23 && tma)
    k_particles<2, 0, 23, 23, 1, kStreamable><<<nblocks, kPushThreads, smem, st>>>(P);
  else if (D == 2 && MODE == 0 && P.t.W[0] == 23 && P.t.W[1] == 15)
    k_particles<2, 0, 23, 15><<<nblocks, kPushThreads, smem, st>>>(P);
  else if (D == 2 && MODE == 0 && P.t.W[0] == 23 && P.t.W[1] == 23)
    k_particles<2, 0, 23, 23><<<nblocks, kPushThreads, smem, st>>>(P);
  else if (D == 2 && MODE == 0 && P.t.W[0] == 25 && P.t.W[1] == 17)
    k_particles<2, 0, 25, 17><<<nblocks, kPushThreads, smem, st>>>(P);
  else if (tma)
    k_particles<D, MODE, 0, 0, 1, kStreamable><<<nblocks, kPushThreads, smem, st>>>(P);
  else if (D == 3 && MODE == 0 && w3)
    k_particles<3, 0, 13, 13, 9><<<nblocks, kPushThreads, smem, st>>>(P);
  else if (D == 3 && MODE == 3 && w3)
    k_particles<3, 3, 13, 13, 9><<<nblocks, kPushThreads, smem, st>>>(P);
  else if (D == 3 && MODE == 0 && w37)
    k_particles<3, 0, 13, 13, 7><<<nblocks, kPushThreads, smem, st>>>(P);
  else if (D == 3 && MODE == 3 && w37)
    k_particles<3, 3, 13, 13, 7><<<nblocks, kPushThreads, smem, st>>>(P);
  else
    k_particles<D, MODE><<<nblocks, kPushThreads, smem, st>>>(P);
  if ((MODE == 0 || MODE == 3) && P.tail_blocks > 0)
    k_particles_tail<D><<<(unsigned)P.tail_blocks, kPushThreads, 0, st>>>(P);
  if (deferred) k_particles_deferred<D, MODE><<<4 * 152, kPushThreads, 0, st>>>(P);
  return cudaSuccess;
}

cudaError_t launch_particles(int dim, int mode, const PushParams& P, cudaStream_t st) {
  if ((long long)P.t.ntiles * P.splits == 0) return cudaSuccess;
  if (mode == 0 && P.wall > 0) mode = 3;  // the fused kernel with the conducting wall
  cudaError_t e;
  switch (dim * 4 + mode) {
    case 4: e = launch<1, 0>(P, st); break;
    case 5: e = launch<1, 1>(P, st); break;
    case 6: e = launch<1, 2>(P, st); break;
    case 7: e = launch<1, 3>(P, st); break;
    case 8: e = launch<2, 0>(P, st); break;
    case 9: e = launch<2, 1>(P, st); break;
    case 10: e = launch<2, 2>(P, st); break;
    case 11: e = launch<2, 3>(P, st); break;
    case 12: e = launch<3, 0>(P, st); break;
    case 13: e = launch<3, 1>(P, st); break;
    case 14: e = launch<3, 2>(P, st); break;
    case 15: e = launch<3, 3>(P, st); break;
    default: return cudaErrorInvalidValue;
  }
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace pic
