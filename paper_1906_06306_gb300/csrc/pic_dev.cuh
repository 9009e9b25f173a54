// Device-side building blocks of the PIC step (arXiv:1906.06306): lattice
// indexing, field accessors, linear gather, Boris push, position update and
// ZigZag current.  Everything is FP32 in cell-relative coordinates: a particle
// is (int cell, float offset in [0,1) per gridded axis), so the arithmetic of
// gather and deposit never sees the absolute position.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace pic {

enum { EX = 0, EY, EZ, BX, BY, BZ, JX, JY, JZ };

// device status word bits (pic_check)
enum : int {
  ST_BAD_CELL = 1,
  ST_BAD_OFF = 2,
  ST_BAD_U = 4,
  ST_BEHIND_WALL = 8,
  ST_TIMEOUT = 16,
  ST_BAD_BUCKETS = 32  // bucket starts handed in were not a partition of the particles
};

// ---- bulk asynchronous copies (TMA engine) and shared-memory barriers ----
// Hand-written PTX for sm_90+: a 1D cp.async.bulk copy from global to shared
// memory completes on an mbarrier with a transaction count of its bytes.

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
// makes the initialised barriers visible to the copy engine (then a block barrier)
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(
                   smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(
                   smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of `parity` to complete, for at most about a second of
// SM clock (2^31 cycles), and with a status word, no longer than until
// another wait has timed out; false when it gave up, having set ST_TIMEOUT in
// the status word (the caller stops using the barrier).
constexpr long long kWaitCycles = 1LL << 31;
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int* status) {
  if (mbar_test(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_test(bar, parity)) {
    const bool others = status && (*reinterpret_cast<volatile int*>(status) & ST_TIMEOUT);
    if (others || clock64() - t0 > kWaitCycles) {
      if (status) atomicOr(status, ST_TIMEOUT);
      return false;
    }
  }
  return true;
}
// box of a 3D tensor map at coordinates (x, y, z) into dst (128-byte aligned),
// completing on bar; the map lives in kernel parameter space
__device__ __forceinline__ void tensor_load_3d(void* dst, const void* map, int x, int y, int z,
                                               unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}
// orders this thread's earlier generic-proxy accesses of shared memory before
// later async-proxy (bulk copy) writes to it: a stage is re-filled by a copy
// only after every thread has read it
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// bytes (a multiple of 16) from src to dst (both 16-byte aligned), completing
// on bar
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes,
                                          unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

struct GridDev {
  int dim;
  int n[3];          // cells per axis (1 for non-gridded axes)
  long long plane;   // n0*n1*n2
  float c;           // Courant number
  int order;         // spatial order of the field solver: 2 (FDTD2) or 4 (FDTD4)
};

struct TileDev {
  int T[3];    // cells per tile (1 on non-gridded axes)
  int nt[3];   // tiles per axis
  int H;       // halo staged on the low side; H+1 on the high side
  int W[3];    // window extent T + 2H + 1 (1 on non-gridded axes)
  int wcells;   // W0*W1*W2
  int wstride;  // wcells rounded up to a multiple of 4 (16-byte aligned planes)
  int ntiles;
  int S[3];     // sub-tile extents: the sort orders a tile's particles by sub-tile
  int ns[3];    // sub-tiles per tile along each axis
  int nsub;     // sub-tiles per tile (sort bins per tile)
};

struct SpeciesDev {
  float q;            // macro-particle charge
  float qm;           // q/m, the s-hat of Appendix C
  long long n;        // particles
  long long ld;       // row length of the SoA arrays (capacity, >= n)
  long long tail;     // particles [tail, n) were appended since the last sort
  int* cell;          // particle arrays written by the push
  float* off;         // [D][ld]
  float* u;           // [3][ld]
  const int* rcell;   // particle arrays read by the push (the sorted buffer right
  const float* roff;  // after a sort inside the step, else the same as cell/off/u)
  const float* ru;
  const int* tstart;  // [ntiles+1] tile bucket offsets
  int* cell_old;      // pre-move snapshot (split gather/deposit path)
  float* off_old;     // [D][ld]
  int* dlist;         // particles deferred to the global-memory pass (room for ld):
                      // stencil outside the tile window, or a move across the wall
  int* dcount;        // entries in dlist
};

// Exact division of 0 <= x < 2^31 by a fixed divisor d >= 1 by multiply and
// shift (Granlund and Montgomery, 1994): with l = ceil(log2 d), s = 31 + l and
// M = ceil(2^s / d) < 2^32, floor(x / d) = (x * M) >> s.  M exceeds 2^s / d by
// less than 1, so x M / 2^s exceeds x / d by less than x / 2^s < 2^-l <= 1/d,
// which cannot carry the fractional part of x / d (at most 1 - 1/d) past 1.
struct FastDiv {
  unsigned long long M;
  int s;
  int d;
};

__device__ __forceinline__ int fdiv(int x, const FastDiv& f) {
  return (int)(((unsigned long long)(unsigned)x * f.M) >> f.s);
}

__device__ __forceinline__ int wrapi(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// Lanes below this one in its warp, as a bit mask.
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Periodic image of a lattice index that is at most one period away.
__device__ __forceinline__ int wrap1(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Shared-memory window of a tile: 6 field components then Jx, Jy, Jz, each a
// W0 x W1 x W2 block, x fastest.  Indices are window-local.
struct SmemAcc {
  float* s;
  int W0, W01, wcells;
  __device__ __forceinline__ float ld(int comp, int i, int j, int k) const {
    return s[comp * wcells + i + W0 * j + W01 * k];
  }
  __device__ __forceinline__ void add(int comp, int i, int j, int k, float v) const {
    atomicAdd(&s[comp * wcells + i + W0 * j + W01 * k], v);
  }
};

// Shared-memory current window in int32 fixed point: the caller passes values
// already divided by the quantum; integer shared atomics are native (FP32 ones
// retry in a loop when lanes collide).  Planes Jx, Jy, Jz of W0 x W1 x W2 ints.
// 2D shared-memory ZigZag with both segments in FP32x2 registers
// (zigzag_smem2 below)
#ifndef PIC_ZZ_PACKED
#define PIC_ZZ_PACKED 1
#endif
// the same for the 3D shared-memory ZigZag (zigzag_smem3)
#ifndef PIC_ZZ_PACKED3
#define PIC_ZZ_PACKED3 1
#endif
#ifndef PIC_MAGIC_F2I
#define PIC_MAGIC_F2I 1
#endif
struct SmemJ {
  int* ji;
  int W0, W01, wc;
  __device__ __forceinline__ void add(int comp, int i, int j, int k, float v) const {
#if PIC_MAGIC_F2I
    // round to nearest integer by adding 1.5 * 2^23 (exact for |v| < 2^22, which
    // the quantum guarantees for a single term) and reading the low mantissa
    const int iv = __float_as_int(v + 12582912.0f) - 0x4B400000;
#else
    const int iv = __float2int_rn(v);
#endif
    atomicAdd(&ji[(comp - JX) * wc + i + W0 * j + W01 * k], iv);
  }
};

// 2D shared-memory current window with two int32 fixed-point words per 64-bit
// shared atomic.  Three planes of 64-bit words, indexed by the lower corner c
// of a ZigZag segment's cell (x fastest, row length W0):
//   Q[c] = (Jx(i,j),   Jy(i,j))
//   R[c] = (Jx(i,j+1), Jy(i+1,j))
//   P[c] = (Jz(i,j),   Jz(i+1,j))        (row j+1 goes to P[c + W0])
// so a segment's 8 words take 4 atomics.  A pair (a, b) of quantised values
// is the integer b 2^32 + a: the low word's sign borrows from the high word,
// so sums of pairs stay exact as long as each word's sum fits in int32, and
// lo = (int32) S, hi = (S - lo) >> 32 recover both.  The pair is formed by one
// packed add of 1.5 * 2^23 (rounding each value to an integer, as SmemJ does)
// and one 64-bit subtract of the two biases.
struct SmemJ64 {
  unsigned long long* Q;  // P = Q + 2 ws, R = Q + ws
  int W0, ws;
  __device__ __forceinline__ static unsigned long long pair(float a, float b) {
    const float2 t = __fadd2_rn(make_float2(a, b), make_float2(12582912.0f, 12582912.0f));
    const unsigned long long bits =
        ((unsigned long long)__float_as_uint(t.y) << 32) | __float_as_uint(t.x);
    return bits - 0x4B4000004B400000ULL;
  }
  // the 8 words of zz_values<2> for a segment in the cell with corner I
  __device__ __forceinline__ void deposit(const int* I, const float* v) const {
    const int c = I[0] + W0 * I[1];
    atomicAdd(&Q[c], pair(v[0], v[2]));
    atomicAdd(&Q[ws + c], pair(v[1], v[3]));
    atomicAdd(&Q[2 * ws + c], pair(v[4], v[5]));
    atomicAdd(&Q[2 * ws + c + W0], pair(v[6], v[7]));
  }
  __device__ __forceinline__ static int lo(unsigned long long s) { return (int)(unsigned)s; }
  __device__ __forceinline__ static int hi(unsigned long long s) {
    return (int)((long long)(s - (unsigned long long)(long long)lo(s)) >> 32);
  }
};

// Global field planes with periodic wrap; indices are lattice indices that may
// lie up to one period outside [0, n).
struct GlobAcc {
  float* F;
  long long plane;
  int n0, n1, n2;
  __device__ __forceinline__ long long at(int i, int j, int k) const {
    return (long long)wrapi(i, n0) + (long long)n0 * (wrapi(j, n1) + (long long)n1 * wrapi(k, n2));
  }
  __device__ __forceinline__ float ld(int comp, int i, int j, int k) const {
    return __ldg(&F[comp * plane + at(i, j, k)]);
  }
  __device__ __forceinline__ void add(int comp, int i, int j, int k, float v) const {
    atomicAdd(&F[comp * plane + at(i, j, k)], v);
  }
};

// Linear interpolation (LinearInterpolator, Sect. 2.3.2) of one staggered
// component.  `stag` has bit d set when the component sits half a cell up axis
// d (Sect. 2.3.1); b is the particle's cell in accessor coordinates, o its
// offsets.  A half-staggered axis uses the lattice points below/above x - 1/2.
template <int D, class Acc>
__device__ __forceinline__ float interp1(const Acc& A, int comp, int stag, const int* b,
                                         const float* o) {
  int i0[3] = {0, 0, 0};
  float w[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int d = 0; d < D; ++d) {
    if (stag & (1 << d)) {
      const bool up = o[d] >= 0.5f;
      i0[d] = up ? b[d] : b[d] - 1;
      w[d] = up ? o[d] - 0.5f : o[d] + 0.5f;
    } else {
      i0[d] = b[d];
      w[d] = o[d];
    }
  }
  if (D == 1) {
    const float f0 = A.ld(comp, i0[0], 0, 0), f1 = A.ld(comp, i0[0] + 1, 0, 0);
    return fmaf(w[0], f1 - f0, f0);
  } else if (D == 2) {
    const float f00 = A.ld(comp, i0[0], i0[1], 0), f10 = A.ld(comp, i0[0] + 1, i0[1], 0);
    const float f01 = A.ld(comp, i0[0], i0[1] + 1, 0), f11 = A.ld(comp, i0[0] + 1, i0[1] + 1, 0);
    const float a = fmaf(w[0], f10 - f00, f00), c = fmaf(w[0], f11 - f01, f01);
    return fmaf(w[1], c - a, a);
  } else {
    float r[2];
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      const int k = i0[2] + kk;
      const float f00 = A.ld(comp, i0[0], i0[1], k), f10 = A.ld(comp, i0[0] + 1, i0[1], k);
      const float f01 = A.ld(comp, i0[0], i0[1] + 1, k), f11 = A.ld(comp, i0[0] + 1, i0[1] + 1, k);
      const float a = fmaf(w[0], f10 - f00, f00), c = fmaf(w[0], f11 - f01, f01);
      r[kk] = fmaf(w[1], c - a, a);
    }
    return fmaf(w[2], r[1] - r[0], r[0]);
  }
}

// E and B at the particle: Ex (1/2,0,0) Ey (0,1/2,0) Ez (0,0,1/2)
// Bx (0,1/2,1/2) By (1/2,0,1/2) Bz (1/2,1/2,0).
template <int D, class Acc>
__device__ __forceinline__ void gather(const Acc& A, const int* b, const float* o, float* e,
                                       float* bf) {
  e[0] = interp1<D>(A, EX, 1, b, o);
  e[1] = interp1<D>(A, EY, 2, b, o);
  e[2] = interp1<D>(A, EZ, 4, b, o);
  bf[0] = interp1<D>(A, BX, 6, b, o);
  bf[1] = interp1<D>(A, BY, 5, b, o);
  bf[2] = interp1<D>(A, BZ, 3, b, o);
}

// Relativistic Boris scheme, Appendix C: u1 = c u + (s/2) E,
// gamma1 = sqrt(1 + u1^2/c^2), t = s B / (2 c gamma1), f = 2/(1 + t^2),
// u2 = f (u1 + u1 x t), u3 = u1 + u2 x t + (s/2) E, u <- u3 / c.
// Evaluated in units of u (every step divided by c, which drops the scalings
// by c): k = s / (2 c), u1 = u + k E, gamma1 = sqrt(1 + u1^2),
// t = k B / gamma1, v = f (u1 + u1 x t), u <- u1 + v x t + k E.
// 1/gamma1 and f use the hardware reciprocal square root and fast divide
// (a few ulp; far inside the FP32-vs-FP64 tolerance).
__device__ __forceinline__ void boris(float* u, const float* e, const float* b, float qm, float c,
                                      float inv_c, float inv_c2) {
  (void)c;
  (void)inv_c2;
  const float k = 0.5f * qm * inv_c;
  float ke[3], u1[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    ke[a] = k * e[a];
    u1[a] = u[a] + ke[a];
  }
  const float ig1 = rsqrtf(fmaf(u1[0], u1[0], fmaf(u1[1], u1[1], fmaf(u1[2], u1[2], 1.0f))));
  const float tf = k * ig1;
  const float t0 = tf * b[0], t1 = tf * b[1], t2 = tf * b[2];
  const float f = __fdividef(2.0f, fmaf(t0, t0, fmaf(t1, t1, fmaf(t2, t2, 1.0f))));
  const float v0 = f * (u1[0] + (u1[1] * t2 - u1[2] * t1));
  const float v1 = f * (u1[1] + (u1[2] * t0 - u1[0] * t2));
  const float v2 = f * (u1[2] + (u1[0] * t1 - u1[1] * t0));
  u[0] = (u1[0] + (v1 * t2 - v2 * t1)) + ke[0];
  u[1] = (u1[1] + (v2 * t0 - v0 * t2)) + ke[1];
  u[2] = (u1[2] + (v0 * t1 - v1 * t0)) + ke[2];
}

// Higuera-Cary pusher (Table 2; Higuera and Cary 2017): the Boris steps with
// the rotation's Lorentz factor gamma+ solved from
// gamma+^2 = (sigma + sqrt(sigma^2 + 4 a)) / 2, sigma = gamma1^2 - tau^2,
// a = tau^2 + (u1 . tau / c)^2, tau = s B / (2 c); for sigma < 0 the same root
// is evaluated as 2 a / (sqrt(sigma^2 + 4 a) - sigma), free of cancellation.
// The rotation is the implicit midpoint um = (u1 + (u1.t) t + u1 x t)/(1 + t^2)
// with t = tau / gamma+, then u3 = um + um x t + (s/2) E.  Keeps the E x B drift
// exact at any speed.
__device__ __forceinline__ void higuera_cary(float* u, const float* e, const float* b, float qm,
                                             float c, float inv_c, float inv_c2) {
  const float hs = 0.5f * qm;
  float u1[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) u1[a] = fmaf(c, u[a], hs * e[a]);
  const float g2 = fmaf(u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2], inv_c2, 1.0f);
  const float tf = hs * inv_c;
  const float ta = tf * b[0], tb = tf * b[1], tc = tf * b[2];
  const float tt = fmaf(ta, ta, fmaf(tb, tb, tc * tc));
  const float us = (u1[0] * ta + u1[1] * tb + u1[2] * tc) * inv_c;
  const float sigma = g2 - tt;
  const float a4 = 4.0f * fmaf(us, us, tt);
  const float r = sqrtf(fmaf(sigma, sigma, a4));
  const float gp2 = sigma >= 0.0f ? 0.5f * (sigma + r) : __fdividef(0.5f * a4, r - sigma);
  const float ig = rsqrtf(gp2);
  const float t0 = ta * ig, t1 = tb * ig, t2 = tc * ig;
  const float sf = __fdividef(1.0f, fmaf(t0, t0, fmaf(t1, t1, fmaf(t2, t2, 1.0f))));
  const float ut = u1[0] * t0 + u1[1] * t1 + u1[2] * t2;
  const float m0 = sf * (fmaf(ut, t0, u1[0]) + (u1[1] * t2 - u1[2] * t1));
  const float m1 = sf * (fmaf(ut, t1, u1[1]) + (u1[2] * t0 - u1[0] * t2));
  const float m2 = sf * (fmaf(ut, t2, u1[2]) + (u1[0] * t1 - u1[1] * t0));
  u[0] = (m0 + (m1 * t2 - m2 * t1) + hs * e[0]) * inv_c;
  u[1] = (m1 + (m2 * t0 - m0 * t2) + hs * e[1]) * inv_c;
  u[2] = (m2 + (m0 * t1 - m1 * t0) + hs * e[2]) * inv_c;
}

// Position update of Eq. (fdX), x += c u / gamma, on the offsets, with every
// operation correctly rounded and none contracted, so the cell bookkeeping can
// be replayed bit for bit: gamma = sqrt(((1 + ux^2) + uy^2) + uz^2),
// r = 1 / gamma, dx = (c u) r, o2 = o1 + dx; o2 < 0 moves one cell down
// (o2 += 1), o2 >= 1 one cell up (o2 -= 1); an o2 + 1 that rounds to 1 is the
// lower cell face, so the particle stays with offset 0.  dn receives dx of
// every axis.
template <int D>
__device__ __forceinline__ void move(const float* u, const float* o1, float c, float* o2, int* dc,
                                     float* dn) {
  const float g2 = __fadd_rn(__fadd_rn(__fadd_rn(1.0f, __fmul_rn(u[0], u[0])), __fmul_rn(u[1], u[1])),
                             __fmul_rn(u[2], u[2]));
  const float r = __frcp_rn(__fsqrt_rn(g2));
#pragma unroll
  for (int a = 0; a < 3; ++a) dn[a] = __fmul_rn(__fmul_rn(c, u[a]), r);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    float o = __fadd_rn(o1[d], dn[d]);
    int k = 0;
    if (o < 0.0f) {
      o = __fadd_rn(o, 1.0f);
      k = -1;
      if (o >= 1.0f) {
        o = 0.0f;
        k = 0;
      }
    } else if (o >= 1.0f) {
      o = __fadd_rn(o, -1.0f);
      k = 1;
    }
    o2[d] = o;
    dc[d] = k;
  }
}

// Number of current words one ZigZag segment touches in D dimensions.
template <int D>
__host__ __device__ constexpr int zz_words() {
  return D == 1 ? 5 : D == 2 ? 8 : 12;
}

// Values that one ZigZag segment (Appendix D) adds to its current words: flux
// q*Dl, weights W (segment midpoint minus the lower corner of its cell).  A
// current component goes to its cell's index along its own axis and is split
// (1-W, W) along every other gridded axis.  In 3D the transverse product is the
// average along the straight segment, midpoint product +- Dl_b Dl_c / 12,
// which keeps the first-order charge exactly conserved.  Order of the words:
//   1D: Jx(i) Jy(i) Jy(i+1) Jz(i) Jz(i+1)
//   2D: Jx(i,j) Jx(i,j+1) Jy(i,j) Jy(i+1,j) Jz(i,j) Jz(i+1,j) Jz(i,j+1) Jz(i+1,j+1)
//   3D: Jx at (i, j+{0,1}, k+{0,1}), Jy at (i+{0,1}, j, k+{0,1}),
//       Jz at (i+{0,1}, j+{0,1}, k), second index fastest in each group
template <int D>
__device__ __forceinline__ void zz_values(const float* Dl, const float* W, float q, float* v) {
  const float f0 = q * Dl[0], f1 = q * Dl[1], f2 = q * Dl[2];
  if (D == 1) {
    v[0] = f0;
    v[1] = f1 * (1.0f - W[0]);
    v[2] = f1 * W[0];
    v[3] = f2 * (1.0f - W[0]);
    v[4] = f2 * W[0];
  } else if (D == 2) {
    const float wx = W[0], wy = W[1], mx = 1.0f - W[0], my = 1.0f - W[1];
    v[0] = f0 * my;
    v[1] = f0 * wy;
    v[2] = f1 * mx;
    v[3] = f1 * wx;
    v[4] = f2 * (mx * my);
    v[5] = f2 * (wx * my);
    v[6] = f2 * (mx * wy);
    v[7] = f2 * (wx * wy);
  } else {
    const float wx = W[0], wy = W[1], wz = W[2];
    const float mx = 1.0f - wx, my = 1.0f - wy, mz = 1.0f - wz;
    const float cyz = Dl[1] * Dl[2] * (1.0f / 12.0f);
    const float czx = Dl[2] * Dl[0] * (1.0f / 12.0f);
    const float cxy = Dl[0] * Dl[1] * (1.0f / 12.0f);
    v[0] = f0 * (my * mz + cyz);
    v[1] = f0 * (wy * mz - cyz);
    v[2] = f0 * (my * wz - cyz);
    v[3] = f0 * (wy * wz + cyz);
    v[4] = f1 * (mz * mx + czx);
    v[5] = f1 * (wz * mx - czx);
    v[6] = f1 * (mz * wx - czx);
    v[7] = f1 * (wz * wx + czx);
    v[8] = f2 * (mx * my + cxy);
    v[9] = f2 * (wx * my - cxy);
    v[10] = f2 * (mx * wy - cxy);
    v[11] = f2 * (wx * wy + cxy);
  }
}

// Add the words of zz_values for a segment in the cell with lower corner I.
template <int D, class Acc>
__device__ __forceinline__ void zz_deposit(const Acc& A, const int* I, const float* v) {
  if (D == 1) {
    A.add(JX, I[0], 0, 0, v[0]);
    A.add(JY, I[0], 0, 0, v[1]);
    A.add(JY, I[0] + 1, 0, 0, v[2]);
    A.add(JZ, I[0], 0, 0, v[3]);
    A.add(JZ, I[0] + 1, 0, 0, v[4]);
  } else if (D == 2) {
    A.add(JX, I[0], I[1], 0, v[0]);
    A.add(JX, I[0], I[1] + 1, 0, v[1]);
    A.add(JY, I[0], I[1], 0, v[2]);
    A.add(JY, I[0] + 1, I[1], 0, v[3]);
    A.add(JZ, I[0], I[1], 0, v[4]);
    A.add(JZ, I[0] + 1, I[1], 0, v[5]);
    A.add(JZ, I[0], I[1] + 1, 0, v[6]);
    A.add(JZ, I[0] + 1, I[1] + 1, 0, v[7]);
  } else {
    A.add(JX, I[0], I[1], I[2], v[0]);
    A.add(JX, I[0], I[1] + 1, I[2], v[1]);
    A.add(JX, I[0], I[1], I[2] + 1, v[2]);
    A.add(JX, I[0], I[1] + 1, I[2] + 1, v[3]);
    A.add(JY, I[0], I[1], I[2], v[4]);
    A.add(JY, I[0], I[1], I[2] + 1, v[5]);
    A.add(JY, I[0] + 1, I[1], I[2], v[6]);
    A.add(JY, I[0] + 1, I[1], I[2] + 1, v[7]);
    A.add(JZ, I[0], I[1], I[2], v[8]);
    A.add(JZ, I[0] + 1, I[1], I[2], v[9]);
    A.add(JZ, I[0], I[1] + 1, I[2], v[10]);
    A.add(JZ, I[0] + 1, I[1] + 1, I[2], v[11]);
  }
}

// ZigZag current of one move (Appendix D), in coordinates relative to the
// lower corner b of the old cell: x1 = o1, x2 = dc + o2 on gridded axes; the
// relay point x_r = min(min(0, dc) + 1, max(max(0, dc), (x1 + x2)/2)); the
// segments carry x_r - x1 and x2 - x_r with weights (x1 + x_r)/2 and
// (x2 + x_r)/2 - dc.  A non-gridded axis moves by dn, split evenly.  When the
// particle stays in its cell both segments add to the same words, so their
// values are summed first and only particles that crossed a face issue the
// second set of atomics.
//
// The 2D shared-memory window path evaluates both segments at once with the
// packed FP32x2 instructions, each register pair holding (segment 1,
// segment 2) of one quantity, so no operand needs a lane swap: the relay
// point is x_r = max(dc, 0) on an axis the move crossed and the midpoint
// otherwise (the min/max above in those two cases), and the word values are
// zz_values<2>'s products.
__device__ __forceinline__ void zigzag_smem2(const SmemJ& A, const int* b, const int* dc,
                                             const float* o1, const float* o2, const float* dn,
                                             float q) {
  float2 Dp[3], Wp[2];
  bool crossed = false;
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    const float x1 = o1[d];
    const float kf = (float)dc[d];
    const float x2 = kf + o2[d];
    const float xr = dc[d] != 0 ? fmaxf(kf, 0.0f) : 0.5f * (x1 + x2);
    const float2 P = make_float2(x1, xr), Q = make_float2(xr, x2);
    Dp[d] = __fadd2_rn(Q, make_float2(-P.x, -P.y));
    Wp[d] = __ffma2_rn(make_float2(0.5f, 0.5f), __fadd2_rn(P, Q), make_float2(0.0f, -kf));
    crossed |= dc[d] != 0;
  }
  Dp[2] = make_float2(0.5f * dn[2], 0.5f * dn[2]);
  const float2 q2 = make_float2(q, q), one = make_float2(1.0f, 1.0f);
  const float2 fx = __fmul2_rn(q2, Dp[0]), fy = __fmul2_rn(q2, Dp[1]), fz = __fmul2_rn(q2, Dp[2]);
  const float2 mx = __fadd2_rn(one, make_float2(-Wp[0].x, -Wp[0].y));
  const float2 my = __fadd2_rn(one, make_float2(-Wp[1].x, -Wp[1].y));
  const float2 fzmy = __fmul2_rn(fz, my), fzwy = __fmul2_rn(fz, Wp[1]);
  float2 v[8] = {__fmul2_rn(fx, my),   __fmul2_rn(fx, Wp[1]), __fmul2_rn(fy, mx),
                 __fmul2_rn(fy, Wp[0]), __fmul2_rn(fzmy, mx), __fmul2_rn(fzmy, Wp[0]),
                 __fmul2_rn(fzwy, mx), __fmul2_rn(fzwy, Wp[0])};
  if (!crossed) {
#pragma unroll
    for (int w = 0; w < 8; ++w) v[w].x += v[w].y;
  }
  // both segments' words rounded to the fixed-point quantum at once
  int i1[8], i2[8];
#pragma unroll
  for (int w = 0; w < 8; ++w) {
#if PIC_MAGIC_F2I
    const float2 t = __fadd2_rn(v[w], make_float2(12582912.0f, 12582912.0f));
    i1[w] = __float_as_int(t.x) - 0x4B400000;
    i2[w] = __float_as_int(t.y) - 0x4B400000;
#else
    i1[w] = __float2int_rn(v[w].x);
    i2[w] = __float2int_rn(v[w].y);
#endif
  }
  // words in the order of zz_deposit<2>: Jx(i,j) Jx(i,j+1) Jy(i,j) Jy(i+1,j)
  // Jz(i,j) Jz(i+1,j) Jz(i,j+1) Jz(i+1,j+1)
  auto put = [&](int bi, int bj, const int* iv) {
    int* J = A.ji + bi + A.W0 * bj;
    atomicAdd(J, iv[0]);
    atomicAdd(J + A.W0, iv[1]);
    atomicAdd(J + A.wc, iv[2]);
    atomicAdd(J + A.wc + 1, iv[3]);
    atomicAdd(J + 2 * A.wc, iv[4]);
    atomicAdd(J + 2 * A.wc + 1, iv[5]);
    atomicAdd(J + 2 * A.wc + A.W0, iv[6]);
    atomicAdd(J + 2 * A.wc + A.W0 + 1, iv[7]);
  };
  put(b[0], b[1], i1);
  if (crossed) put(b[0] + dc[0], b[1] + dc[1], i2);
}

// The 3D shared-memory window path in the same way: both segments' relay
// points, displacements and weights as (segment 1, segment 2) pairs, and
// zz_values<3>'s twelve products, with the +-D_b D_c / 12 terms, evaluated on
// the pairs; the words of a segment in zz_deposit<3>'s order.
__device__ __forceinline__ void zigzag_smem3(const SmemJ& A, const int* b, const int* dc,
                                             const float* o1, const float* o2, float q) {
  float2 Dp[3], Wp[3], Mp[3];
  bool crossed = false;
  const float2 one = make_float2(1.0f, 1.0f);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float x1 = o1[d];
    const float kf = (float)dc[d];
    const float x2 = kf + o2[d];
    const float xr = dc[d] != 0 ? fmaxf(kf, 0.0f) : 0.5f * (x1 + x2);
    const float2 P = make_float2(x1, xr), Q = make_float2(xr, x2);
    Dp[d] = __fadd2_rn(Q, make_float2(-P.x, -P.y));
    Wp[d] = __ffma2_rn(make_float2(0.5f, 0.5f), __fadd2_rn(P, Q), make_float2(0.0f, -kf));
    Mp[d] = __fadd2_rn(one, make_float2(-Wp[d].x, -Wp[d].y));
    crossed |= dc[d] != 0;
  }
  const float2 q2 = make_float2(q, q), c12 = make_float2(1.0f / 12.0f, 1.0f / 12.0f);
  const float2 f0 = __fmul2_rn(q2, Dp[0]), f1 = __fmul2_rn(q2, Dp[1]), f2 = __fmul2_rn(q2, Dp[2]);
  const float2 cyz = __fmul2_rn(__fmul2_rn(Dp[1], Dp[2]), c12);
  const float2 czx = __fmul2_rn(__fmul2_rn(Dp[2], Dp[0]), c12);
  const float2 cxy = __fmul2_rn(__fmul2_rn(Dp[0], Dp[1]), c12);
  const float2 nyz = make_float2(-cyz.x, -cyz.y), nzx = make_float2(-czx.x, -czx.y),
               nxy = make_float2(-cxy.x, -cxy.y);
  const float2 &wx = Wp[0], &wy = Wp[1], &wz = Wp[2], &mx = Mp[0], &my = Mp[1], &mz = Mp[2];
  float2 v[12] = {__fmul2_rn(f0, __ffma2_rn(my, mz, cyz)),  __fmul2_rn(f0, __ffma2_rn(wy, mz, nyz)),
                  __fmul2_rn(f0, __ffma2_rn(my, wz, nyz)),  __fmul2_rn(f0, __ffma2_rn(wy, wz, cyz)),
                  __fmul2_rn(f1, __ffma2_rn(mz, mx, czx)),  __fmul2_rn(f1, __ffma2_rn(wz, mx, nzx)),
                  __fmul2_rn(f1, __ffma2_rn(mz, wx, nzx)),  __fmul2_rn(f1, __ffma2_rn(wz, wx, czx)),
                  __fmul2_rn(f2, __ffma2_rn(mx, my, cxy)),  __fmul2_rn(f2, __ffma2_rn(wx, my, nxy)),
                  __fmul2_rn(f2, __ffma2_rn(mx, wy, nxy)),  __fmul2_rn(f2, __ffma2_rn(wx, wy, cxy))};
  if (!crossed) {
#pragma unroll
    for (int w = 0; w < 12; ++w) v[w].x += v[w].y;
  }
  int i1[12], i2[12];
#pragma unroll
  for (int w = 0; w < 12; ++w) {
#if PIC_MAGIC_F2I
    const float2 t = __fadd2_rn(v[w], make_float2(12582912.0f, 12582912.0f));
    i1[w] = __float_as_int(t.x) - 0x4B400000;
    i2[w] = __float_as_int(t.y) - 0x4B400000;
#else
    i1[w] = __float2int_rn(v[w].x);
    i2[w] = __float2int_rn(v[w].y);
#endif
  }
  // zz_deposit<3>'s words: Jx at (i, j+{0,1}, k+{0,1}), Jy at (i+{0,1}, j,
  // k+{0,1}), Jz at (i+{0,1}, j+{0,1}, k), second index fastest
  auto put = [&](int bi, int bj, int bk, const int* iv) {
    int* J = A.ji + bi + A.W0 * bj + A.W01 * bk;
    atomicAdd(J, iv[0]);
    atomicAdd(J + A.W0, iv[1]);
    atomicAdd(J + A.W01, iv[2]);
    atomicAdd(J + A.W0 + A.W01, iv[3]);
    atomicAdd(J + A.wc, iv[4]);
    atomicAdd(J + A.wc + A.W01, iv[5]);
    atomicAdd(J + A.wc + 1, iv[6]);
    atomicAdd(J + A.wc + 1 + A.W01, iv[7]);
    atomicAdd(J + 2 * A.wc, iv[8]);
    atomicAdd(J + 2 * A.wc + 1, iv[9]);
    atomicAdd(J + 2 * A.wc + A.W0, iv[10]);
    atomicAdd(J + 2 * A.wc + A.W0 + 1, iv[11]);
  };
  put(b[0], b[1], b[2], i1);
  if (crossed) put(b[0] + dc[0], b[1] + dc[1], b[2] + dc[2], i2);
}

template <int D, class Acc>
__device__ __forceinline__ void zigzag(const Acc& A, const int* b, const int* dc, const float* o1,
                                       const float* o2, const float* dn, float q) {
  if constexpr (D == 2 && PIC_ZZ_PACKED && std::is_same<Acc, SmemJ>::value) {
    zigzag_smem2(A, b, dc, o1, o2, dn, q);
    return;
  }
  if constexpr (D == 3 && PIC_ZZ_PACKED3 && std::is_same<Acc, SmemJ>::value) {
    zigzag_smem3(A, b, dc, o1, o2, q);
    return;
  }
  float D1[3], D2[3], W1[3] = {0.f, 0.f, 0.f}, W2[3] = {0.f, 0.f, 0.f};
  int b2[3] = {b[0], b[1], b[2]};
  bool crossed = false;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (d < D) {
      const float x1 = o1[d];
      const float x2 = (float)dc[d] + o2[d];
      const float lo = (float)(dc[d] < 0 ? dc[d] : 0) + 1.0f;
      const float hi = (float)(dc[d] > 0 ? dc[d] : 0);
      const float xr = fminf(lo, fmaxf(hi, 0.5f * (x1 + x2)));
      D1[d] = xr - x1;
      D2[d] = x2 - xr;
      W1[d] = 0.5f * (x1 + xr);
      W2[d] = 0.5f * (x2 + xr) - (float)dc[d];
      b2[d] = b[d] + dc[d];
      crossed |= dc[d] != 0;
    } else {
      D1[d] = 0.5f * dn[d];
      D2[d] = D1[d];
    }
  }
  float v1[zz_words<D>()], v2[zz_words<D>()];
  zz_values<D>(D1, W1, q, v1);
  zz_values<D>(D2, W2, q, v2);
  if (!crossed) {
#pragma unroll
    for (int w = 0; w < zz_words<D>(); ++w) v1[w] += v2[w];
  }
  if constexpr (std::is_same<Acc, SmemJ64>::value) {
    A.deposit(b, v1);
    if (crossed) A.deposit(b2, v2);
  } else {
    zz_deposit<D>(A, b, v1);
    if (crossed) zz_deposit<D>(A, b2, v2);
  }
}

}  // namespace pic
