// Discrete adjoint (reverse mode) of the PIC step of arXiv:1906.06306 (FDTD2
// field solver, Boris pusher, periodic box): the gradient of a loss with
// respect to the state before a step from its gradient with respect to the
// state after it.  The step is
//   B1 = B - (c/2) curl+ E;  e, b = gather(E, B1; x);  u' = Boris(u, e, b)
//   x' = x + c u'/gamma(u');  J = sum ZigZag(x, x');  B2 = B1 - (c/2) curl+ E
//   E' = E + c curl- B2 - F^p J
// On the periodic lattice (curl+)^T = curl- and (curl-)^T = curl+, and the
// Binomial2 filter is symmetric, so the field part is two stencil kernels
// and the filter; the particle part is the chain rule through gather, Boris,
// move and ZigZag for every particle, one thread each (the cell of a particle
// and the branch of the ZigZag relay point are locally constant, so they are
// taken from the forward step).  Particles grouped by tile (given the bucket
// starts of the sort that grouped them) go through k_adj_tiles: a block stages
// its tile window of E, B and the current adjoint in shared memory and sums
// the field adjoints there (int32 fixed point), and the particles whose
// stencil left the window are deferred to the global-memory pass; ungrouped
// particles all take the global-memory pass.
#include <cmath>

#include "pic_kernels.h"

namespace pic {

// Adjoint of E' = E + c curl- B2 - Jf:  Bbar += c curl+ Ebar,  Jbar = -Ebar.
template <int D>
__global__ void k_adj_e(float* __restrict__ A, const GridDev g, float c) {
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const long long P = g.plane;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n0) return;
  FOR_ROWS(j, k) {
    const long long idx = (long long)i + (long long)n0 * (j + (long long)n1 * k);
    const long long sx = (i + 1 < n0) ? 1 : 1 - n0;
    const long long sy = (D >= 2) ? ((j + 1 < n1) ? n0 : (long long)n0 * (1 - n1)) : 0;
    const long long sz = (D >= 3) ? ((k + 1 < n2) ? (long long)n0 * n1 : (long long)n0 * n1 * (1 - n2)) : 0;
    const float* Ex = A + EX * P;
    const float* Ey = A + EY * P;
    const float* Ez = A + EZ * P;
    const float ex = Ex[idx], ey = Ey[idx], ez = Ez[idx];
    float cx = 0.f, cy = 0.f, cz = 0.f;
    cy -= Ez[idx + sx] - ez;
    cz += Ey[idx + sx] - ey;
    if (D >= 2) {
      cx += Ez[idx + sy] - ez;
      cz -= Ex[idx + sy] - ex;
    }
    if (D >= 3) {
      cx -= Ey[idx + sz] - ey;
      cy += Ex[idx + sz] - ex;
    }
    A[BX * P + idx] += c * cx;
    A[BY * P + idx] += c * cy;
    A[BZ * P + idx] += c * cz;
    A[JX * P + idx] = -ex;
    A[JY * P + idx] = -ey;
    A[JZ * P + idx] = -ez;
  }
}

// Adjoint of B <- B - h curl+ E (a half step, h = c/2):  Ebar -= h curl- Bbar.
// Reads only B planes and writes only E planes, so the points are independent.
template <int D>
__global__ void k_adj_b(float* __restrict__ A, const GridDev g, float h) {
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const long long P = g.plane;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n0) return;
  FOR_ROWS(j, k) {
    const long long idx = (long long)i + (long long)n0 * (j + (long long)n1 * k);
    const long long sx = (i > 0) ? 1 : 1 - n0;
    const long long sy = (D >= 2) ? ((j > 0) ? n0 : (long long)n0 * (1 - n1)) : 0;
    const long long sz = (D >= 3) ? ((k > 0) ? (long long)n0 * n1 : (long long)n0 * n1 * (1 - n2)) : 0;
    const float* Bx = A + BX * P;
    const float* By = A + BY * P;
    const float* Bz = A + BZ * P;
    const float bx = Bx[idx], by = By[idx], bz = Bz[idx];
    float cx = 0.f, cy = 0.f, cz = 0.f;
    cy -= bz - Bz[idx - sx];
    cz += by - By[idx - sx];
    if (D >= 2) {
      cx += bz - Bz[idx - sy];
      cz -= bx - Bx[idx - sy];
    }
    if (D >= 3) {
      cx -= by - By[idx - sz];
      cy += bx - Bx[idx - sz];
    }
    A[EX * P + idx] -= h * cx;
    A[EY * P + idx] -= h * cy;
    A[EZ * P + idx] -= h * cz;
  }
}

// Reverse of the linear gather of one staggered component (stag bit d: half a
// cell up axis d): Abar[comp] += weights * vb (atomic), xb += dvalue/dx * vb.
template <int D, class AF, class AB>
__device__ __forceinline__ void gather_adj(const AF& F, const AB& Ab, int comp, int stag,
                                           const int* b, const float* o, float vb, float* xb) {
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
#pragma unroll
  for (int cn = 0; cn < (1 << D); ++cn) {
    const int oc[3] = {cn & 1, (cn >> 1) & 1, (cn >> 2) & 1};
    float wt = 1.f;
#pragma unroll
    for (int d = 0; d < D; ++d) wt *= oc[d] ? w[d] : 1.f - w[d];
    const int ii = i0[0] + oc[0], jj = D >= 2 ? i0[1] + oc[1] : 0, kk = D >= 3 ? i0[2] + oc[2] : 0;
    Ab.add(comp, ii, jj, kk, wt * vb);
    const float f = F.ld(comp, ii, jj, kk) * vb;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      float dw = oc[d] ? 1.f : -1.f;
#pragma unroll
      for (int d2 = 0; d2 < D; ++d2)
        if (d2 != d) dw *= oc[d2] ? w[d2] : 1.f - w[d2];
      xb[d] += dw * f;
    }
  }
}

__device__ __forceinline__ void cross3(const float* a, const float* b, float* r) {
  r[0] = a[1] * b[2] - a[2] * b[1];
  r[1] = a[2] * b[0] - a[0] * b[2];
  r[2] = a[0] * b[1] - a[1] * b[0];
}

// Reverse of the Boris push (Appendix C) u' = u3/c: u1 = c u + hs e,
// g1 = (1 + u1^2/c^2)^(-1/2), t = (hs/c) g1 b, f = 2/(1 + t^2),
// v = f (u1 + u1 x t), u3 = u1 + v x t + hs e.  From ub' (gradient of u'),
// the gradients ub, eb, bb of u, e, b.
__device__ __forceinline__ void boris_adj(const float* u, const float* e, const float* b, float qm,
                                          float c, const float* upb, float* ub, float* eb,
                                          float* bb) {
  const float hs = 0.5f * qm;
  float u1[3], t[3], s[3], v[3], x[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) u1[a] = fmaf(c, u[a], hs * e[a]);
  const float ic2 = 1.0f / (c * c);
  const float g1 = rsqrtf(fmaf(u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2], ic2, 1.0f));
  const float tf = hs / c * g1;
#pragma unroll
  for (int a = 0; a < 3; ++a) t[a] = tf * b[a];
  const float f = 2.0f / fmaf(t[0], t[0], fmaf(t[1], t[1], fmaf(t[2], t[2], 1.0f)));
  cross3(u1, t, x);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    s[a] = u1[a] + x[a];
    v[a] = f * s[a];
  }
  float u3b[3], u1b[3], vb[3], tb[3], sb[3], tmp[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    u3b[a] = upb[a] / c;
    u1b[a] = u3b[a];
    eb[a] = hs * u3b[a];
  }
  cross3(t, u3b, vb);  // w = v x t
  cross3(u3b, v, tb);
  float fb = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    fb = fmaf(vb[a], s[a], fb);
    sb[a] = f * vb[a];
  }
  cross3(t, sb, tmp);  // s = u1 + u1 x t
#pragma unroll
  for (int a = 0; a < 3; ++a) u1b[a] += sb[a] + tmp[a];
  cross3(sb, u1, tmp);
  const float denb = -0.5f * f * f * fb;  // f = 2 / (1 + t.t)
#pragma unroll
  for (int a = 0; a < 3; ++a) tb[a] += tmp[a] + 2.0f * t[a] * denb;
  float tfb = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    tfb = fmaf(tb[a], b[a], tfb);
    bb[a] = tf * tb[a];
  }
  const float g1b = tfb * hs / c;  // tf = (hs/c) g1, dg1/du1 = -g1^3 u1 / c^2
  const float k = -g1b * g1 * g1 * g1 * ic2;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    u1b[a] = fmaf(k, u1[a], u1b[a]);
    ub[a] = c * u1b[a];
    eb[a] = fmaf(hs, u1b[a], eb[a]);
  }
}

// Reverse of one ZigZag segment's words (the forward zz_values / zz_deposit,
// Appendix D) in the cell with lower corner I: from Jbar, the gradients of the
// segment displacement Dl and of its weights W.
template <int D, class AB>
__device__ __forceinline__ void segment_adj(const AB& Ab, const int* I, float q,
                                            const float* Dl, const float* W, float* Db,
                                            float* Wb) {
  const int i = I[0], j = I[1], k = I[2];
  const float f0 = q * Dl[0], f1 = q * Dl[1], f2 = q * Dl[2];
  if (D == 1) {
    const float x0 = Ab.ld(JX, i, 0, 0);
    const float y0 = Ab.ld(JY, i, 0, 0), y1 = Ab.ld(JY, i + 1, 0, 0);
    const float z0 = Ab.ld(JZ, i, 0, 0), z1 = Ab.ld(JZ, i + 1, 0, 0);
    const float wx = W[0], mx = 1.f - wx;
    Db[0] += q * x0;
    Db[1] += q * (mx * y0 + wx * y1);
    Db[2] += q * (mx * z0 + wx * z1);
    Wb[0] += f1 * (y1 - y0) + f2 * (z1 - z0);
  } else if (D == 2) {
    const float x00 = Ab.ld(JX, i, j, 0), x01 = Ab.ld(JX, i, j + 1, 0);
    const float y00 = Ab.ld(JY, i, j, 0), y10 = Ab.ld(JY, i + 1, j, 0);
    const float z00 = Ab.ld(JZ, i, j, 0), z10 = Ab.ld(JZ, i + 1, j, 0);
    const float z01 = Ab.ld(JZ, i, j + 1, 0), z11 = Ab.ld(JZ, i + 1, j + 1, 0);
    const float wx = W[0], wy = W[1], mx = 1.f - wx, my = 1.f - wy;
    Db[0] += q * (my * x00 + wy * x01);
    Db[1] += q * (mx * y00 + wx * y10);
    Db[2] += q * (mx * my * z00 + wx * my * z10 + mx * wy * z01 + wx * wy * z11);
    Wb[0] += f1 * (y10 - y00) + f2 * (my * (z10 - z00) + wy * (z11 - z01));
    Wb[1] += f0 * (x01 - x00) + f2 * (mx * (z01 - z00) + wx * (z11 - z10));
  } else {
    // each component: words at (second, third) corner offsets 00 10 01 11 of
    // its two transverse axes (b, c) = (a+1, a+2) mod 3, weights
    // (1-Wb or Wb)(1-Wc or Wc) +- Db Dc / 12
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int bx = (a + 1) % 3, cx = (a + 2) % 3;
      float J00, J10, J01, J11;  // offsets along (b, c)
      int o00[3] = {i, j, k}, o10[3] = {i, j, k}, o01[3] = {i, j, k}, o11[3] = {i, j, k};
      o10[bx] += 1;
      o01[cx] += 1;
      o11[bx] += 1;
      o11[cx] += 1;
      J00 = Ab.ld(JX + a, o00[0], o00[1], o00[2]);
      J10 = Ab.ld(JX + a, o10[0], o10[1], o10[2]);
      J01 = Ab.ld(JX + a, o01[0], o01[1], o01[2]);
      J11 = Ab.ld(JX + a, o11[0], o11[1], o11[2]);
      const float wb = W[bx], wc = W[cx], mb = 1.f - wb, mc = 1.f - wc;
      const float cc = Dl[bx] * Dl[cx] * (1.0f / 12.0f);
      const float fa = q * Dl[a];
      Db[a] += q * ((mb * mc + cc) * J00 + (wb * mc - cc) * J10 + (mb * wc - cc) * J01 +
                    (wb * wc + cc) * J11);
      Wb[bx] += fa * (mc * (J10 - J00) + wc * (J11 - J01));
      Wb[cx] += fa * (mb * (J01 - J00) + wb * (J11 - J10));
      const float sgn = fa * (J00 - J10 - J01 + J11) * (1.0f / 12.0f);
      Db[bx] += sgn * Dl[cx];
      Db[cx] += sgn * Dl[bx];
    }
    (void)f0;
    (void)f1;
    (void)f2;
  }
}

// Reverse of the particle update of particle p of species S, in cell b
// (accessor coordinates of F and Ab), up to the gather: the forward gather,
// Boris and move are recomputed with the forward kernel's own routines, then
// ZigZag, move and Boris are reversed.  ubar of p is updated in place; out:
// the offsets o1, the position gradient so far xb, and the particle's E and B
// adjoints ebb (Ex, Ey, Ez, Bx, By, Bz), which the caller takes back through
// the gather (gather_adj).
template <int D, class AF, class AB>
__device__ __forceinline__ void adj_chain(const AF& F, const AB& Ab, const AdjSpecies& S,
                                          long long p, const int* b, float c, float* o1,
                                          float* xb, float* ebb) {
  const long long ld = S.ld;
  float u[3];
  o1[0] = o1[1] = o1[2] = 0.f;
#pragma unroll
  for (int d = 0; d < D; ++d) o1[d] = S.off[d * ld + p];
#pragma unroll
  for (int a = 0; a < 3; ++a) u[a] = S.u[a * ld + p];
  // forward: gather, Boris, move (the forward kernel's own routines)
  float e[3], bf[3];
  gather<D>(F, b, o1, e, bf);
  float u2[3] = {u[0], u[1], u[2]};
  boris(u2, e, bf, S.qm, c, 1.0f / c, 1.0f / (c * c));
  float o2[3] = {0.f, 0.f, 0.f}, dn[3];
  int dc[3] = {0, 0, 0};
  move<D>(u2, o1, c, o2, dc, dn);
  const float g2 = fmaf(u2[0], u2[0], fmaf(u2[1], u2[1], fmaf(u2[2], u2[2], 1.0f)));
  const float ig = rsqrtf(g2);
  // reverse of x' = x + dn: xbar passes through, dn gets xbar
  float dnb[3] = {0.f, 0.f, 0.f}, u2b[3];
  xb[0] = xb[1] = xb[2] = 0.f;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    xb[d] = S.xbar[d * ld + p];
    dnb[d] = xb[d];
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) u2b[a] = S.ubar[a * ld + p];
  // reverse of ZigZag(x, x + dn), positions relative to the old cell
  float D1[3], D2[3], W1[3] = {0.f, 0.f, 0.f}, W2[3] = {0.f, 0.f, 0.f};
  bool mid[3] = {false, false, false};
  int b2[3] = {b[0], b[1], b[2]};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (d < D) {
      const float x1 = o1[d], x2 = (float)dc[d] + o2[d];
      const float lo = (float)(dc[d] < 0 ? dc[d] : 0) + 1.0f;
      const float hi = (float)(dc[d] > 0 ? dc[d] : 0);
      const float m = 0.5f * (x1 + x2);
      const float xr = fminf(lo, fmaxf(hi, m));
      mid[d] = m > hi && m < lo;
      D1[d] = xr - x1;
      D2[d] = x2 - xr;
      W1[d] = 0.5f * (x1 + xr);
      W2[d] = 0.5f * (x2 + xr) - (float)dc[d];
      b2[d] = b[d] + dc[d];
    } else {
      D1[d] = D2[d] = 0.5f * dn[d];
    }
  }
  float D1b[3] = {0.f, 0.f, 0.f}, D2b[3] = {0.f, 0.f, 0.f};
  float W1b[3] = {0.f, 0.f, 0.f}, W2b[3] = {0.f, 0.f, 0.f};
  segment_adj<D>(Ab, b, S.q, D1, W1, D1b, W1b);
  segment_adj<D>(Ab, b2, S.q, D2, W2, D2b, W2b);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (d < D) {
      const float xrb = D1b[d] - D2b[d] + 0.5f * (W1b[d] + W2b[d]);
      float x1b = -D1b[d] + 0.5f * W1b[d];
      float x2b = D2b[d] + 0.5f * W2b[d];
      if (mid[d]) {
        x1b += 0.5f * xrb;
        x2b += 0.5f * xrb;
      }
      xb[d] += x1b + x2b;  // x2 = x1 + dn
      dnb[d] += x2b;
    } else {
      dnb[d] += 0.5f * (D1b[d] + D2b[d]);
    }
  }
  // reverse of dn = c u2 / gamma
  const float ud = u2[0] * dnb[0] + u2[1] * dnb[1] + u2[2] * dnb[2];
#pragma unroll
  for (int a = 0; a < 3; ++a) u2b[a] += c * ig * (dnb[a] - u2[a] * ud * ig * ig);
  float ub[3];
  boris_adj(u, e, bf, S.qm, c, u2b, ub, ebb, ebb + 3);
#pragma unroll
  for (int a = 0; a < 3; ++a) S.ubar[a * ld + p] = ub[a];
}

// Stagger bits of the six components: Ex (1/2,0,0) Ey (0,1/2,0) Ez (0,0,1/2)
// Bx (0,1/2,1/2) By (1/2,0,1/2) Bz (1/2,1/2,0).
__device__ constexpr int kStagger[6] = {1, 2, 4, 6, 5, 3};

// The whole reverse for one particle through global memory: the chain, then
// the gather's reverse with the field adjoints added through Ab; xbar of p
// is written.
template <int D, class AF, class AB>
__device__ __forceinline__ void adj_particle(const AF& F, const AB& Ab, const AdjSpecies& S,
                                             long long p, const int* b, float c) {
  float o1[3], xb[3], ebb[6];
  adj_chain<D>(F, Ab, S, p, b, c, o1, xb, ebb);
#pragma unroll
  for (int comp = 0; comp < 6; ++comp)
    gather_adj<D>(F, Ab, EX + comp, kStagger[comp], b, o1, ebb[comp], xb);
#pragma unroll
  for (int d = 0; d < D; ++d) S.xbar[d * S.ld + p] = xb[d];
}

// The lattice cell (i, j, k) of a linear cell index.
__device__ __forceinline__ void cell_ijk(const AdjParams& P, int cell, int* b) {
  const int r = fdiv(cell, P.div0);
  b[0] = cell - r * P.g.n[0];
  b[2] = fdiv(r, P.div1);
  b[1] = r - b[2] * P.g.n[1];
}

// Global-memory pass: every particle of every species, or (deferred) the
// particles listed by k_adj_tiles.
template <int D>
__global__ void __launch_bounds__(256) k_adj_particles(const AdjParams P, int deferred) {
  const GlobAcc F{const_cast<float*>(P.F1), P.g.plane, P.g.n[0], P.g.n[1], P.g.n[2]};
  const GlobAcc Ab{P.A, P.g.plane, P.g.n[0], P.g.n[1], P.g.n[2]};
  const float c = P.g.c;
  for (int s = 0; s < P.nspecies; ++s) {
    const AdjSpecies& S = P.sp[s];
    const long long n = deferred ? (long long)P.dcount[s] : S.n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
      const long long p = deferred ? (long long)S.dlist[i] : i;
      const int cell = S.cell[p];
      if (cell < 0 || (long long)cell >= P.g.plane) continue;
      int b[3];
      cell_ijk(P, cell, b);
      adj_particle<D>(F, Ab, S, p, b, c);
    }
  }
}

// The tile window of the adjoint pass in shared memory, window-local
// coordinates: planes 0..5 forward E and B1, 6..8 the current adjoint.  One
// accessor serves as both the forward fields and the adjoint planes; it adds
// nothing: the tile pass takes each particle's E and B adjoints and adds
// them itself.
struct AdjWin {
  const float* S;
  int W0, W01, ws;
  __device__ __forceinline__ int at(int i, int j, int k) const { return i + W0 * j + W01 * k; }
  __device__ __forceinline__ float ld(int comp, int i, int j, int k) const {
    return S[comp * ws + at(i, j, k)];
  }
  __device__ __forceinline__ void add(int, int, int, int, float) const {}
};

// Window geometry of block (tile, split) of a tile pass.
struct AdjBlock {
  int tile, split;
  int w0[3], W[3];
};
template <int D>
__device__ __forceinline__ AdjBlock adj_block(const AdjParams& P) {
  const TileDev& t = P.t;
  AdjBlock B;
  B.tile = blockIdx.x / P.splits;
  B.split = blockIdx.x % P.splits;
  const int tc[3] = {B.tile % t.nt[0], (B.tile / t.nt[0]) % t.nt[1], B.tile / (t.nt[0] * t.nt[1])};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    B.w0[d] = d < D ? tc[d] * t.T[d] - t.H : 0;
    B.W[d] = d < D ? t.W[d] : 1;
  }
  return B;
}
// Window-local cell of a particle and whether its stencil (cells b - 1 ..
// b + 2 on every gridded axis, as in the forward tile kernel) is inside the
// window.
template <int D>
__device__ __forceinline__ bool adj_in_window(const AdjParams& P, const AdjBlock& B, int cell,
                                              int* l) {
  int ijk[3];
  cell_ijk(P, cell, ijk);
  bool inwin = true;
  l[0] = l[1] = l[2] = 0;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    l[d] = wrapi(ijk[d] - B.w0[d], P.g.n[d]);
    inwin &= (unsigned)(l[d] - 1) <= (unsigned)(B.W[d] - 4);
  }
  return inwin;
}
// This block's share [a, b) of species s's tile bucket.
__device__ __forceinline__ void adj_share(const AdjParams& P, const AdjSpecies& S,
                                          const AdjBlock& B, long long& a, long long& b) {
  const long long lo = S.tstart[B.tile * P.t.nsub], hi = S.tstart[(B.tile + 1) * P.t.nsub];
  a = lo + (hi - lo) * B.split / P.splits;
  b = lo + (hi - lo) * (B.split + 1) / P.splits;
}

// The tile pass (particles grouped by tile): one block per (tile, split)
// stages its window of E, B1 and the current adjoint and runs its share of
// each species' bucket, in batches of 256, through the reverse chain, reading
// the fields there.  The particles' E and B adjoints go back through the
// transposed gather (weights times the value, the stencils of gather_adj)
// onto the window as int32 fixed point: native integer shared-memory atomics
// (an FP32 shared atomic is a retry loop, which lanes sharing a word turn into
// a queue).  The quantum is set per batch from the batch's largest magnitude
// M (a block reduction): q = 2^(e - 22) with M < 2^e, so one term is below
// 2^22 quanta and a batch (at most one term per particle and word) below
// 2^30; after every batch the integers are folded into an FP32 window, which
// goes to the lattice once per window cell.  A particle whose stencil is not
// inside the window goes on the species' deferred list for the global pass.
template <int D>
__global__ void __launch_bounds__(256, D == 3 ? 2 : PIC_ADJ_MIN_BLOCKS)
    k_adj_tiles(const AdjParams P) {
  extern __shared__ __align__(16) float sm[];
  __shared__ unsigned wmax[8];  // per warp of the block (256 threads)
  const AdjBlock B = adj_block<D>(P);
  const int wc = P.t.wcells, ws = P.t.wstride;
  const long long plane = P.g.plane;
  const GlobAcc G{P.A, plane, P.g.n[0], P.g.n[1], P.g.n[2]};
  int* wi = reinterpret_cast<int*>(sm + 9 * ws);  // 6 planes of fixed-point sums
  float* wf = sm + 15 * ws;                       // 6 planes of their FP32 folds
  for (int w = threadIdx.x; w < wc; w += blockDim.x) {
    const int lx = w % B.W[0], rr = w / B.W[0], ly = rr % B.W[1], lz = rr / B.W[1];
    const long long gi = G.at(B.w0[0] + lx, B.w0[1] + ly, B.w0[2] + lz);
#pragma unroll
    for (int c = 0; c < 6; ++c) sm[c * ws + w] = __ldg(&P.F1[c * plane + gi]);
#pragma unroll
    for (int a = 0; a < 3; ++a) sm[(6 + a) * ws + w] = P.A[(JX + a) * plane + gi];
  }
  for (int w = threadIdx.x; w < 6 * ws; w += blockDim.x) {
    wi[w] = 0;
    wf[w] = 0.f;
  }
  __syncthreads();
  const AdjWin WN{sm, B.W[0], B.W[0] * B.W[1], ws};
  const int W0 = B.W[0], W01 = B.W[0] * B.W[1];
  const float c = P.g.c;
  for (int s = 0; s < P.nspecies; ++s) {
    const AdjSpecies& S = P.sp[s];
    if (S.n == 0) continue;
    long long a, b;
    adj_share(P, S, B, a, b);
    const long long ld = S.ld;
    for (long long base = a; base < b; base += blockDim.x) {  // the same count for every thread
      const long long p = base + threadIdx.x;
      float ebb[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, o[3] = {0.f, 0.f, 0.f}, xb[3];
      int l[3] = {0, 0, 0};
      bool mine = false;
      if (p < b) {
        const int cell = S.cell[p];
        if (cell >= 0 && (long long)cell < plane) {
          if (adj_in_window<D>(P, B, cell, l)) {
            adj_chain<D>(WN, WN, S, p, l, c, o, xb, ebb);
            mine = true;
          } else {
            S.dlist[atomicAdd(&P.dcount[s], 1)] = (int)p;
          }
        }
      }
      // the batch's largest magnitude (non-negative floats order as their bits)
      float m = 0.f;
#pragma unroll
      for (int k = 0; k < 6; ++k) m = fmaxf(m, fabsf(ebb[k]));
      const unsigned mw = __reduce_max_sync(0xffffffffu, __float_as_uint(m));
      if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mw;
      __syncthreads();
      unsigned mb = 0u;
#pragma unroll
      for (int k = 0; k < 8; ++k) mb = max(mb, wmax[k]);
      const float M = __uint_as_float(mb);
      int e = 0;
      frexpf(M, &e);  // M < 2^e
      const float q = ldexpf(1.0f, e - 22), inv_q = ldexpf(1.0f, 22 - e);
      if (mine) {
        // the gather's reverse (gather_adj's operations, in its order, for the
        // position gradient) with each term also added, in quanta, to the window
#pragma unroll
        for (int comp = 0; comp < 6; ++comp) {
          const float vb = ebb[comp], v = vb * inv_q;
          int i0[3] = {0, 0, 0};
          float w[3] = {0.f, 0.f, 0.f};
#pragma unroll
          for (int d = 0; d < D; ++d) {
            if (kStagger[comp] & (1 << d)) {
              const bool up = o[d] >= 0.5f;
              i0[d] = up ? l[d] : l[d] - 1;
              w[d] = up ? o[d] - 0.5f : o[d] + 0.5f;
            } else {
              i0[d] = l[d];
              w[d] = o[d];
            }
          }
#pragma unroll
          for (int cn = 0; cn < (1 << D); ++cn) {
            const int oc[3] = {cn & 1, (cn >> 1) & 1, (cn >> 2) & 1};
            float wt = 1.f;
#pragma unroll
            for (int d = 0; d < D; ++d) wt *= oc[d] ? w[d] : 1.f - w[d];
            const int at = (i0[0] + oc[0]) + W0 * (i0[1] + oc[1]) + W01 * (i0[2] + oc[2]);
            atomicAdd(&wi[comp * ws + at], __float2int_rn(wt * v));
            const float f = sm[(EX + comp) * ws + at] * vb;
#pragma unroll
            for (int d = 0; d < D; ++d) {
              float dw = oc[d] ? 1.f : -1.f;
#pragma unroll
              for (int d2 = 0; d2 < D; ++d2)
                if (d2 != d) dw *= oc[d2] ? w[d2] : 1.f - w[d2];
              xb[d] += dw * f;
            }
          }
        }
#pragma unroll
        for (int d = 0; d < D; ++d) S.xbar[d * ld + p] = xb[d];
      }
      __syncthreads();
      if (mb != 0u) {
        for (int w = threadIdx.x; w < 6 * ws; w += blockDim.x) {
          const int v = wi[w];
          if (v != 0) {
            wf[w] += (float)v * q;
            wi[w] = 0;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int w = threadIdx.x; w < wc; w += blockDim.x) {
    const int lx = w % B.W[0], rr = w / B.W[0], ly = rr % B.W[1], lz = rr / B.W[1];
    const long long gi = G.at(B.w0[0] + lx, B.w0[1] + ly, B.w0[2] + lz);
#pragma unroll
    for (int c2 = 0; c2 < 6; ++c2) {
      const float v = wf[c2 * ws + w];
      if (v != 0.f) atomicAdd(&P.A[c2 * plane + gi], v);
    }
  }
}

cudaError_t launch_adj_e(const GridDev& g, float* A, cudaStream_t st) {
  const RowLaunch L = row_launch(g);
  switch (g.dim) {
    case 1: k_adj_e<1><<<L.grid, L.threads, 0, st>>>(A, g, g.c); break;
    case 2: k_adj_e<2><<<L.grid, L.threads, 0, st>>>(A, g, g.c); break;
    case 3: k_adj_e<3><<<L.grid, L.threads, 0, st>>>(A, g, g.c); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_adj_b_half(const GridDev& g, float* A, cudaStream_t st) {
  const RowLaunch L = row_launch(g);
  const float h = 0.5f * g.c;
  switch (g.dim) {
    case 1: k_adj_b<1><<<L.grid, L.threads, 0, st>>>(A, g, h); break;
    case 2: k_adj_b<2><<<L.grid, L.threads, 0, st>>>(A, g, h); break;
    case 3: k_adj_b<3><<<L.grid, L.threads, 0, st>>>(A, g, h); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// shared memory of the tile pass: 9 float planes (E, B1, current adjoint),
// 6 int32 and 6 float planes (the E and B adjoint sums)
size_t adj_tile_smem_bytes(const TileDev& t) { return sizeof(float) * 21 * (size_t)t.wstride; }

cudaError_t launch_adj_particles(const AdjParams& P, cudaStream_t st) {
  long long nmax = 0;
  for (int s = 0; s < P.nspecies; ++s) nmax = P.sp[s].n > nmax ? P.sp[s].n : nmax;
  if (nmax == 0) return cudaSuccess;
  // the tile pass when every species with particles has its tile grouping
  bool tiled = true;
  for (int s = 0; s < P.nspecies; ++s) tiled &= P.sp[s].n == 0 || P.sp[s].tstart != nullptr;
  tiled &= adj_tile_smem_bytes(P.t) <= 200 * 1024;  // else the window does not fit
  const int D = P.g.dim;
  if (tiled) {
    static bool attr[4] = {false, false, false, false};
    const size_t smem = adj_tile_smem_bytes(P.t);
    cudaError_t e = cudaMemsetAsync(P.dcount, 0, sizeof(int) * P.nspecies, st);
    if (e != cudaSuccess) return e;
    if (!attr[D]) {
      const void* k1 = D == 1 ? (const void*)k_adj_tiles<1> : D == 2 ? (const void*)k_adj_tiles<2>
                                                                      : (const void*)k_adj_tiles<3>;
      e = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      if (e != cudaSuccess) return e;
      attr[D] = true;
    }
    const long long blocks = (long long)P.t.ntiles * P.splits;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    switch (D) {
      case 1: k_adj_tiles<1><<<(unsigned)blocks, 256, smem, st>>>(P); break;
      case 2: k_adj_tiles<2><<<(unsigned)blocks, 256, smem, st>>>(P); break;
      case 3: k_adj_tiles<3><<<(unsigned)blocks, 256, smem, st>>>(P); break;
      default: return cudaErrorInvalidValue;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // the global pass: every particle, or those the tile pass deferred (their
  // count is on the device: a grid that strides over any count)
  long long nb = tiled ? 152LL * 8 : (nmax + 255) / 256;
  if (nb > 152LL * 32) nb = 152LL * 32;
  const int deferred = tiled ? 1 : 0;
  switch (D) {
    case 1: k_adj_particles<1><<<(unsigned)nb, 256, 0, st>>>(P, deferred); break;
    case 2: k_adj_particles<2><<<(unsigned)nb, 256, 0, st>>>(P, deferred); break;
    case 3: k_adj_particles<3><<<(unsigned)nb, 256, 0, st>>>(P, deferred); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace pic
