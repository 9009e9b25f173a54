/* FP64 CPU oracle of the relativistic PIC time step (arXiv:1906.06306).
 * TEST INFRASTRUCTURE ONLY: see pic_oracle.h.  Plain loops, periodic wrap by
 * modulo on every access, no blocking or fusion; each function follows the
 * passage of the paper named in its comment. */
#include "pic_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

enum { EX, EY, EZ, BX, BY, BZ, JX, JY, JZ };

static long wrapi(long i, long n) {
  long r = i % n;
  return r < 0 ? r + n : r;
}

static long ncell(const orc_grid* g) { return (long)g->nx * g->ny * g->nz; }

/* flat index of lattice point (i, j, k), periodic in every dimension */
static long at(const orc_grid* g, long i, long j, long k) {
  return (wrapi(k, g->nz) * g->ny + wrapi(j, g->ny)) * g->nx + wrapi(i, g->nx);
}

static double val(const orc_grid* g, const double* F, int comp, long i, long j, long k) {
  return F[comp * ncell(g) + at(g, i, j, k)];
}

/* A(p + e_d) - A(p): the forward difference of Appendix B (nabla^+); zero
 * along a dimension that is not gridded. */
static double dplus(const orc_grid* g, const double* F, int comp, int d, long i, long j, long k) {
  if (d >= g->dim) return 0.0;
  return val(g, F, comp, i + (d == 0), j + (d == 1), k + (d == 2)) - val(g, F, comp, i, j, k);
}

/* A(p) - A(p - e_d): the backward difference of Appendix B (nabla^-). */
static double dminus(const orc_grid* g, const double* F, int comp, int d, long i, long j, long k) {
  if (d >= g->dim) return 0.0;
  return val(g, F, comp, i, j, k) - val(g, F, comp, i - (d == 0), j - (d == 1), k - (d == 2));
}

/* Spatial order of the field solver: 2 (FDTD2, Eqs. fdE/fdB) or 4 (FDTD4 of
 * Table 2, read as the fourth-order staggered difference
 * (9/8) [A(p+e/2) - A(p-e/2)] - (1/24) [A(p+3e/2) - A(p-3e/2)]). */
static int g_order = 2;
void orc_set_field_order(int order) { g_order = order; }

/* forward difference at the point half a cell up axis d, of the chosen order */
static double dplus_o(const orc_grid* g, const double* F, int comp, int d, long i, long j, long k) {
  if (g_order == 2 || d >= g->dim) return dplus(g, F, comp, d, i, j, k);
  const long di = d == 0, dj = d == 1, dk = d == 2;
  const double near = val(g, F, comp, i + di, j + dj, k + dk) - val(g, F, comp, i, j, k);
  const double far = val(g, F, comp, i + 2 * di, j + 2 * dj, k + 2 * dk) -
                     val(g, F, comp, i - di, j - dj, k - dk);
  return 9.0 / 8.0 * near - 1.0 / 24.0 * far;
}

/* backward difference at the point half a cell down axis d, of the chosen order */
static double dminus_o(const orc_grid* g, const double* F, int comp, int d, long i, long j, long k) {
  if (g_order == 2 || d >= g->dim) return dminus(g, F, comp, d, i, j, k);
  const long di = d == 0, dj = d == 1, dk = d == 2;
  const double near = val(g, F, comp, i, j, k) - val(g, F, comp, i - di, j - dj, k - dk);
  const double far = val(g, F, comp, i + di, j + dj, k + dk) -
                     val(g, F, comp, i - 2 * di, j - 2 * dj, k - 2 * dk);
  return 9.0 / 8.0 * near - 1.0 / 24.0 * far;
}

/* Eq. (fdB), half a step.  With E on cell edges and B on faces (Sect. 2.3.1)
 * the curl of E at the B points is taken with forward differences:
 *   (curl E)_x = d+_y Ez - d+_z Ey, (curl E)_y = d+_z Ex - d+_x Ez,
 *   (curl E)_z = d+_x Ey - d+_y Ex. */
void orc_push_half_b(const orc_grid* g, double* F) {
  const long P = ncell(g);
  const double h = 0.5 * g->c;
  for (long k = 0; k < g->nz; ++k)
    for (long j = 0; j < g->ny; ++j)
      for (long i = 0; i < g->nx; ++i) {
        const long p = at(g, i, j, k);
        const double cx = dplus_o(g, F, EZ, 1, i, j, k) - dplus_o(g, F, EY, 2, i, j, k);
        const double cy = dplus_o(g, F, EX, 2, i, j, k) - dplus_o(g, F, EZ, 0, i, j, k);
        const double cz = dplus_o(g, F, EY, 0, i, j, k) - dplus_o(g, F, EX, 1, i, j, k);
        F[BX * P + p] -= h * cx;
        F[BY * P + p] -= h * cy;
        F[BZ * P + p] -= h * cz;
      }
}

/* Curl part of Eq. (fdE): the curl of B at the E points uses backward
 * differences, (curl B)_x = d-_y Bz - d-_z By, and cyclically. */
void orc_push_e(const orc_grid* g, double* F) {
  const long P = ncell(g);
  for (long k = 0; k < g->nz; ++k)
    for (long j = 0; j < g->ny; ++j)
      for (long i = 0; i < g->nx; ++i) {
        const long p = at(g, i, j, k);
        const double cx = dminus_o(g, F, BZ, 1, i, j, k) - dminus_o(g, F, BY, 2, i, j, k);
        const double cy = dminus_o(g, F, BX, 2, i, j, k) - dminus_o(g, F, BZ, 0, i, j, k);
        const double cz = dminus_o(g, F, BY, 0, i, j, k) - dminus_o(g, F, BX, 1, i, j, k);
        F[EX * P + p] += g->c * cx;
        F[EY * P + p] += g->c * cy;
        F[EZ * P + p] += g->c * cz;
      }
}

/* add_cur (Table 1): the -J term of Eq. (fdE). */
void orc_add_cur(const orc_grid* g, double* F) {
  const long P = ncell(g);
  for (int a = 0; a < 3; ++a)
    for (long p = 0; p < P; ++p) F[(EX + a) * P + p] -= F[(JX + a) * P + p];
}

/* Binomial2 (Table 2): the 3-point digital filter (1/4, 1/2, 1/4) applied
 * along each gridded dimension in turn, `passes` times. */
void orc_filter_binomial(const orc_grid* g, double* F, int passes) {
  const long P = ncell(g);
  double* tmp = (double*)malloc(sizeof(double) * P);
  for (int pass = 0; pass < passes; ++pass)
    for (int d = 0; d < g->dim; ++d)
      for (int a = 0; a < 3; ++a) {
        double* J = F + (JX + a) * P;
        memcpy(tmp, J, sizeof(double) * P);
        for (long k = 0; k < g->nz; ++k)
          for (long j = 0; j < g->ny; ++j)
            for (long i = 0; i < g->nx; ++i) {
              const long di = d == 0, dj = d == 1, dk = d == 2;
              J[at(g, i, j, k)] = 0.25 * tmp[at(g, i - di, j - dj, k - dk)] +
                                  0.5 * tmp[at(g, i, j, k)] +
                                  0.25 * tmp[at(g, i + di, j + dj, k + dk)];
            }
      }
  free(tmp);
}

/* Position of each staggered component inside its cell (Sect. 2.3.1). */
static const double STAG[6][3] = {
    {0.5, 0.0, 0.0}, {0.0, 0.5, 0.0}, {0.0, 0.0, 0.5}, /* Ex Ey Ez */
    {0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}, {0.5, 0.5, 0.0}, /* Bx By Bz */
};

/* LinearInterpolator (Sect. 2.3.2, Table 2): each component is weighted from
 * the 2^D lattice points of its own staggered grid that surround x, with the
 * first-order (linear in each dimension) weights. */
void orc_interp(const orc_grid* g, const double* F, const double* x, double* e, double* b) {
  for (int comp = 0; comp < 6; ++comp) {
    long i0[3] = {0, 0, 0};
    double w[3] = {0.0, 0.0, 0.0};
    for (int d = 0; d < g->dim; ++d) {
      const double xi = x[d] - STAG[comp][d];
      i0[d] = (long)floor(xi);
      w[d] = xi - (double)i0[d];
    }
    double s = 0.0;
    for (int c2 = 0; c2 < 2; ++c2)
      for (int c1 = 0; c1 < 2; ++c1)
        for (int c0 = 0; c0 < 2; ++c0) {
          const int o[3] = {c0, c1, c2};
          double wt = 1.0;
          int skip = 0;
          for (int d = 0; d < 3; ++d) {
            if (d >= g->dim) {
              if (o[d]) skip = 1;
            } else {
              wt *= o[d] ? w[d] : 1.0 - w[d];
            }
          }
          if (skip) continue;
          s += wt * val(g, F, comp, i0[0] + c0, i0[1] + c1, i0[2] + c2);
        }
    if (comp < 3)
      e[comp] = s;
    else
      b[comp - 3] = s;
  }
}

static void cross(const double* a, const double* b, double* r) {
  r[0] = a[1] * b[2] - a[2] * b[1];
  r[1] = a[2] * b[0] - a[0] * b[2];
  r[2] = a[0] * b[1] - a[1] * b[0];
}

/* Relativistic Boris scheme, Appendix C, Eqs. (appB1)-(appB2).  Velocities
 * primed there are in units of c:  u1 = c u + s E/2,  gamma1 = sqrt(1 +
 * u1^2/c^2),  t = s B / (2 c gamma1),  f = 2 / (1 + t^2),  u2 = f (u1 + u1 x t),
 * u3 = u1 + u2 x t + s E/2,  u <- u3 / c.  (The rotation keeps |u1|, so the
 * gamma of both half rotations is gamma1; s = q/m enters t.) */
void orc_boris(double* u, const double* e, const double* b, double qm, double c) {
  double u1[3], t[3], u2[3], x1[3], x2[3];
  for (int a = 0; a < 3; ++a) u1[a] = c * u[a] + 0.5 * qm * e[a];
  const double g1 = sqrt(1.0 + (u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]) / (c * c));
  for (int a = 0; a < 3; ++a) t[a] = qm * b[a] / (2.0 * c * g1);
  const double f = 2.0 / (1.0 + t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
  cross(u1, t, x1);
  for (int a = 0; a < 3; ++a) u2[a] = f * (u1[a] + x1[a]);
  cross(u2, t, x2);
  for (int a = 0; a < 3; ++a) u[a] = (u1[a] + x2[a] + 0.5 * qm * e[a]) / c;
}

/* Higuera-Cary (2017): u1 = c u + s E/2 as in Boris; with tau = s B / (2 c),
 * u* = (u1 . tau) / c and sigma = gamma1^2 - tau^2, the rotation uses
 * gamma+ = sqrt((sigma + sqrt(sigma^2 + 4 (tau^2 + u*^2))) / 2) and t = tau / gamma+;
 * the rotated momentum is the implicit midpoint
 * um = (u1 + (u1 . t) t + u1 x t) / (1 + t^2), and u3 = um + um x t + s E/2. */
void orc_higuera_cary(double* u, const double* e, const double* b, double qm, double c) {
  double u1[3], tau[3], t[3], um[3], x1[3], x2[3];
  for (int a = 0; a < 3; ++a) u1[a] = c * u[a] + 0.5 * qm * e[a];
  const double g2 = 1.0 + (u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]) / (c * c);
  for (int a = 0; a < 3; ++a) tau[a] = qm * b[a] / (2.0 * c);
  const double tt = tau[0] * tau[0] + tau[1] * tau[1] + tau[2] * tau[2];
  const double us = (u1[0] * tau[0] + u1[1] * tau[1] + u1[2] * tau[2]) / c;
  const double sigma = g2 - tt;
  const double gp = sqrt(0.5 * (sigma + sqrt(sigma * sigma + 4.0 * (tt + us * us))));
  for (int a = 0; a < 3; ++a) t[a] = tau[a] / gp;
  const double s = 1.0 / (1.0 + t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
  const double ut = u1[0] * t[0] + u1[1] * t[1] + u1[2] * t[2];
  cross(u1, t, x1);
  for (int a = 0; a < 3; ++a) um[a] = s * (u1[a] + ut * t[a] + x1[a]);
  cross(um, t, x2);
  for (int a = 0; a < 3; ++a) u[a] = (um[a] + x2[a] + 0.5 * qm * e[a]) / c;
}

static int g_pusher = 0;
void orc_set_pusher(int pusher) { g_pusher = pusher; }

/* One ZigZag segment: flux Fl from the cell with lower corner I, weights W,
 * displacement Ds of the segment (Appendix D).  Each current component sits
 * half a cell up its own axis (at the E points), so along its own axis it goes
 * to index I; along every other gridded axis it is shared between I and I+1
 * with weights (1 - W, W).
 *
 * In 3D the product of two midpoint weights is not the average of the
 * transverse weight product along the straight segment: the two differ by
 * +-Ds_b Ds_c / 12 (+ when both corner offsets are equal), and without that
 * term the change of the first-order charge misses q Ds_x Ds_y Ds_z / 4 per
 * segment.  Appendices B and D require the deposit to conserve charge, so the
 * term is included in 3D (in 1D and 2D no gridded component has two gridded
 * transverse axes and the midpoint products are exact). */
static int g_abs = 0; /* orc_deposit_abs: add |term| instead of term */
static void deposit_segment(const orc_grid* g, double* F, const long* I, const double* Fl,
                            const double* W, const double* Ds) {
  const long P = ncell(g);
  for (int a = 0; a < 3; ++a)
    for (int c2 = 0; c2 < 2; ++c2)
      for (int c1 = 0; c1 < 2; ++c1)
        for (int c0 = 0; c0 < 2; ++c0) {
          const int o[3] = {c0, c1, c2};
          double wt = 1.0;
          int skip = 0;
          for (int d = 0; d < 3; ++d) {
            if (d >= g->dim || d == a) {
              if (o[d]) skip = 1;
              continue;
            }
            wt *= o[d] ? W[d] : 1.0 - W[d];
          }
          if (skip) continue;
          if (g->dim == 3) {
            const int b = (a + 1) % 3, c = (a + 2) % 3;
            wt += (o[b] == o[c] ? 1.0 : -1.0) * Ds[b] * Ds[c] / 12.0;
          }
          const double v = Fl[a] * wt;
          F[(JX + a) * P + at(g, I[0] + c0, I[1] + c1, I[2] + c2)] += g_abs ? fabs(v) : v;
        }
}

/* ZigZag scheme, Appendix D, Eqs. (appE1)-(appE2): relay point
 * x_r = min(min(i1, i2) + 1, max(max(i1, i2), (x1 + x2)/2)) per gridded
 * dimension with i = floor(x) (the lower lattice index of the particle's cell),
 * fluxes F1 = q (x_r - x1), F2 = q (x2 - x_r), weights W1 = (x1 + x_r)/2 - i1,
 * W2 = (x2 + x_r)/2 - i2.  Along a dimension that is not gridded the relay is
 * the midpoint, so each segment carries half the displacement there. */
void orc_zigzag(const orc_grid* g, double* F, const double* x1, const double* x2, double q) {
  long i1[3] = {0, 0, 0}, i2[3] = {0, 0, 0};
  double xr[3], F1[3], F2[3], D1[3], D2[3], W1[3] = {0, 0, 0}, W2[3] = {0, 0, 0};
  for (int d = 0; d < 3; ++d) {
    if (d < g->dim) {
      i1[d] = (long)floor(x1[d]);
      i2[d] = (long)floor(x2[d]);
      const double lo = (double)(i1[d] < i2[d] ? i1[d] : i2[d]) + 1.0;
      const double hi = (double)(i1[d] > i2[d] ? i1[d] : i2[d]);
      xr[d] = fmin(lo, fmax(hi, 0.5 * (x1[d] + x2[d])));
      W1[d] = 0.5 * (x1[d] + xr[d]) - (double)i1[d];
      W2[d] = 0.5 * (x2[d] + xr[d]) - (double)i2[d];
    } else {
      xr[d] = 0.5 * (x1[d] + x2[d]);
    }
    D1[d] = xr[d] - x1[d];
    D2[d] = x2[d] - xr[d];
    F1[d] = q * D1[d];
    F2[d] = q * D2[d];
  }
  deposit_segment(g, F, i1, F1, W1, D1);
  deposit_segment(g, F, i2, F2, W2, D2);
}

static double extent(const orc_grid* g, int d) { return d == 0 ? g->nx : d == 1 ? g->ny : g->nz; }

/* Conducting wall of the shock set-up (Sect. 4.2) at the node x = g_wall
 * (0: no wall).  See orc_set_wall. */
static long g_wall = 0, g_izero = 0;
void orc_set_wall(long wall, long i_zero) {
  g_wall = wall;
  g_izero = i_zero;
}

/* interp_em and push of Table 1: gather, Boris (Appendix C), then the
 * position update of Eq. (fdX), x += c u / gamma with the new u.  A particle
 * whose new x lies below the wall is reflected specularly: x -> 2 w - x,
 * u_x -> -u_x (the displacement written to dx is the unreflected one; the
 * deposit rebuilds the reflected path from it). */
void orc_push_particles(const orc_grid* g, const double* F, double* x, double* u, long n,
                        double qm, double* x_old, double* dx) {
  for (long p = 0; p < n; ++p) {
    double xp[3] = {0.0, 0.0, 0.0}, e[3], b[3];
    for (int d = 0; d < g->dim; ++d) xp[d] = x[d * n + p];
    orc_interp(g, F, xp, e, b);
    double up[3] = {u[p], u[n + p], u[2 * n + p]};
    if (g_pusher == 1)
      orc_higuera_cary(up, e, b, qm, g->c);
    else
      orc_boris(up, e, b, qm, g->c);
    const double gam = sqrt(1.0 + up[0] * up[0] + up[1] * up[1] + up[2] * up[2]);
    for (int d = 0; d < 3; ++d) {
      u[d * n + p] = up[d];
      dx[d * n + p] = g->c * up[d] / gam;
      x_old[d * n + p] = xp[d];
    }
    for (int d = 0; d < g->dim; ++d) {
      const double L = extent(g, d);
      double xn = xp[d] + dx[d * n + p];
      if (d == 0 && g_wall > 0 && xn < (double)g_wall) {
        xn = 2.0 * (double)g_wall - xn;
        u[p] = -u[p];
      }
      if (xn < 0.0) xn += L;
      if (xn >= L) xn -= L;
      x[d * n + p] = xn;
    }
  }
}

/* comp_curr (Table 1) for one species.  The current of a particle reflected
 * at the wall is deposited along its true path: a straight segment to the
 * point where it meets the wall plane, then the mirrored remainder, each with
 * the ZigZag rule, so the charge moved is accounted for at every node. */
void orc_deposit(const orc_grid* g, double* F, const double* x_old, const double* dx, long n,
                 double q) {
  for (long p = 0; p < n; ++p) {
    double x1[3], x2[3];
    for (int d = 0; d < 3; ++d) {
      x1[d] = x_old[d * n + p];
      x2[d] = x1[d] + dx[d * n + p];
    }
    if (g_wall > 0 && x2[0] < (double)g_wall) {
      const double w = (double)g_wall;
      const double s = (x1[0] - w) / (x1[0] - x2[0]); /* fraction of the step before the wall */
      double xc[3], xm[3];
      xc[0] = w;
      for (int d = 1; d < 3; ++d) xc[d] = x1[d] + s * (x2[d] - x1[d]);
      xm[0] = 2.0 * w - x2[0];
      for (int d = 1; d < 3; ++d) xm[d] = x2[d];
      orc_zigzag(g, F, x1, xc, q);
      orc_zigzag(g, F, xc, xm, q);
    } else {
      orc_zigzag(g, F, x1, x2, q);
    }
  }
}

/* The same deposit with every term of Appendix D's ZigZag sum (one flux times
 * one weight, per current word and segment) added as its absolute value: per
 * word, the sum of |term| over the moves.  It bounds |J| on every word (the
 * triangle inequality) and equals |J| for a single move (all of a move's terms
 * on one component share the sign of its displacement: the weights are
 * non-negative).  FP32 sums the terms in some order, so its rounding error on a
 * word scales with this sum, not with the net J, which can cancel. */
void orc_deposit_abs(const orc_grid* g, double* F, const double* x_old, const double* dx, long n,
                     double q) {
  g_abs = 1;
  orc_deposit(g, F, x_old, dx, n, q);
  g_abs = 0;
}

/* Field boundary of the conducting wall at the node x = w (Sect. 4.2): the
 * tangential E vanishes on the wall plane (Ey = Ez = 0 at i = w) and the cells
 * behind it (i < w) hold the mirror image of the plasma side, the image of a
 * perfect conductor (tangential E and normal B odd, normal E and tangential B
 * even about x = w).  Integer-x components (Ey, Ez, Bx) at i mirror 2w - i;
 * half-integer ones (Ex, By, Bz, stored at i for x = i + 1/2) mirror
 * 2w - 1 - i.  Every E and B value at i >= i_zero is set to zero (the vacuum
 * beyond the injector's last position, which also keeps the periodic wrap from
 * reaching the wall).  J is not touched. */
void orc_wall_fields(const orc_grid* g, double* F, long w, long i_zero) {
  const long P = ncell(g);
  for (long k = 0; k < g->nz; ++k)
    for (long j = 0; j < g->ny; ++j) {
      for (long i = 0; i < w; ++i) {
        const long a = at(g, i, j, k), ri = at(g, 2 * w - i, j, k), rh = at(g, 2 * w - 1 - i, j, k);
        F[EX * P + a] = F[EX * P + rh];
        F[BY * P + a] = F[BY * P + rh];
        F[BZ * P + a] = F[BZ * P + rh];
        F[EY * P + a] = -F[EY * P + ri];
        F[EZ * P + a] = -F[EZ * P + ri];
        F[BX * P + a] = -F[BX * P + ri];
      }
      F[EY * P + at(g, w, j, k)] = 0.0;
      F[EZ * P + at(g, w, j, k)] = 0.0;
      for (long i = i_zero; i < g->nx; ++i)
        for (int comp = EX; comp <= BZ; ++comp) F[comp * P + at(g, i, j, k)] = 0.0;
    }
}

/* Receding injector of the shock set-up (Sect. 4.2).  An upstream template
 * (positions xt[3][nt] in a block [0, lt) x ny x nz, sorted by x; four-
 * velocities ut[3][nt]) is repeated along x (copy m shifted by m lt) and
 * advected at -v_up; the injector sits at X(s) = min(x0 + v_inj s, x_max).
 * In template coordinates the injector is at A(s) = (X(s) - x0) + v_up s, and
 * in step s (ending at time level s + 1) every copy-m particle with
 * A(s) - m lt <= xt < A(s+1) - m lt enters the box at
 * x = xt + ((m lt + x0) - v_up (s + 1)): the particles that crossed the
 * injector during the step.  The new x offset is rounded to float, as every
 * initial offset is (an offset that rounds to 1 moves to the next cell).
 * Writes at most cap particles to xo[3][cap], uo[3][cap] (m ascending, then
 * template order) and returns their count, or -1 if cap is too small. */
static double inj_front(double x0, double x_max, double v_inj, double v_up, long s) {
  const double X = fmin(x0 + v_inj * (double)s, x_max);
  return (X - x0) + v_up * (double)s;
}

long orc_inject(const double* xt, const double* ut, long nt, long lt, double x0, double x_max,
                double v_inj, double v_up, long s, double* xo, double* uo, long cap) {
  const double a = inj_front(x0, x_max, v_inj, v_up, s);
  const double b = inj_front(x0, x_max, v_inj, v_up, s + 1);
  long out = 0;
  for (long m = (long)floor(a / (double)lt); m <= (long)floor(b / (double)lt); ++m) {
    const double am = a - (double)m * (double)lt, bm = b - (double)m * (double)lt;
    const double sh = ((double)m * (double)lt + x0) - v_up * (double)(s + 1);
    for (long k = 0; k < nt; ++k) {
      if (!(xt[k] >= am && xt[k] < bm)) continue;
      if (out >= cap) return -1;
      const double pos = xt[k] + sh;
      double cx = floor(pos);
      double off = (double)(float)(pos - cx);
      if (off == 1.0) {
        cx += 1.0;
        off = 0.0;
      }
      xo[out] = cx + off;
      xo[cap + out] = xt[nt + k];
      xo[2 * cap + out] = xt[2 * nt + k];
      for (int d = 0; d < 3; ++d) uo[d * cap + out] = ut[d * nt + k];
      ++out;
    }
  }
  return out;
}

/* One time step in the order of Table 1 (halo updates are implicit in the
 * periodic indexing; there is a single tile and no MPI). */
void orc_step(const orc_grid* g, double* F, double** x, double** u, const long* n,
              const double* q, const double* m, int ns, int passes, double* work) {
  const long P = ncell(g);
  long o = 0;
  orc_push_half_b(g, F);                               /* push_half_b1 */
  if (g_wall > 0) orc_wall_fields(g, F, g_wall, g_izero);
  for (int s = 0; s < ns; ++s) {                       /* interp_em, push */
    orc_push_particles(g, F, x[s], u[s], n[s], q[s] / m[s], work + o, work + o + 3 * n[s]);
    o += 6 * n[s];
  }
  orc_push_half_b(g, F);                               /* push_half_b2 */
  if (g_wall > 0) orc_wall_fields(g, F, g_wall, g_izero);
  orc_push_e(g, F);                                    /* push_e */
  memset(F + JX * P, 0, sizeof(double) * 3 * P);       /* comp_curr */
  o = 0;
  for (int s = 0; s < ns; ++s) {
    orc_deposit(g, F, work + o, work + o + 3 * n[s], n[s], q[s]);
    o += 6 * n[s];
  }
  orc_filter_binomial(g, F, passes);                   /* Binomial2 on J */
  orc_add_cur(g, F);                                   /* add_cur */
  if (g_wall > 0) orc_wall_fields(g, F, g_wall, g_izero);
}

/* Charge on the nodes with the first-order shape that the ZigZag weights
 * imply (Appendix D): weight 1 - w at floor(x), w at floor(x) + 1. */
void orc_charge_density(const orc_grid* g, const double* x, long n, double q, double* rho) {
  for (long p = 0; p < n; ++p) {
    long i0[3] = {0, 0, 0};
    double w[3] = {0.0, 0.0, 0.0};
    for (int d = 0; d < g->dim; ++d) {
      const double xd = x[d * n + p];
      i0[d] = (long)floor(xd);
      w[d] = xd - (double)i0[d];
    }
    for (int c2 = 0; c2 < 2; ++c2)
      for (int c1 = 0; c1 < 2; ++c1)
        for (int c0 = 0; c0 < 2; ++c0) {
          const int o[3] = {c0, c1, c2};
          double wt = q;
          int skip = 0;
          for (int d = 0; d < 3; ++d) {
            if (d >= g->dim) {
              if (o[d]) skip = 1;
            } else {
              wt *= o[d] ? w[d] : 1.0 - w[d];
            }
          }
          if (!skip) rho[at(g, i0[0] + c0, i0[1] + c1, i0[2] + c2)] += wt;
        }
  }
}

/* Discrete Gauss law operand (Appendix B): backward-difference divergence of
 * E evaluated at the nodes, where the charge lives. */
void orc_div_e(const orc_grid* g, const double* F, double* div) {
  for (long k = 0; k < g->nz; ++k)
    for (long j = 0; j < g->ny; ++j)
      for (long i = 0; i < g->nx; ++i)
        div[at(g, i, j, k)] = dminus(g, F, EX, 0, i, j, k) + dminus(g, F, EY, 1, i, j, k) +
                              dminus(g, F, EZ, 2, i, j, k);
}

/* Forward-difference divergence of B at the cell centres (Appendix B). */
void orc_div_b(const orc_grid* g, const double* F, double* div) {
  for (long k = 0; k < g->nz; ++k)
    for (long j = 0; j < g->ny; ++j)
      for (long i = 0; i < g->nx; ++i)
        div[at(g, i, j, k)] = dplus(g, F, BX, 0, i, j, k) + dplus(g, F, BY, 1, i, j, k) +
                              dplus(g, F, BZ, 2, i, j, k);
}

void orc_field_energy(const orc_grid* g, const double* F, double* out) {
  const long P = ncell(g);
  double se = 0.0, sb = 0.0;
  for (int a = 0; a < 3; ++a)
    for (long p = 0; p < P; ++p) {
      se += F[(EX + a) * P + p] * F[(EX + a) * P + p];
      sb += F[(BX + a) * P + p] * F[(BX + a) * P + p];
    }
  out[0] = 0.5 * se;
  out[1] = 0.5 * sb;
}

/* m c^2 (gamma - 1), with gamma - 1 written as u^2 / (gamma + 1). */
double orc_kinetic_energy(const double* u, long n, double m, double c) {
  double s = 0.0;
  for (long p = 0; p < n; ++p) {
    const double u2 = u[p] * u[p] + u[n + p] * u[n + p] + u[2 * n + p] * u[2 * n + p];
    s += u2 / (sqrt(1.0 + u2) + 1.0);
  }
  return m * c * c * s;
}
