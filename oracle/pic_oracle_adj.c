/* Reverse mode (discrete adjoint) of the oracle's time step: given the
 * gradient of a loss with respect to the state after a step, the gradient
 * with respect to the state before it.  TEST INFRASTRUCTURE ONLY (see
 * pic_oracle.h): plain loops in double precision, FDTD2 field solver, Boris
 * pusher, periodic box.
 *
 * The step (Table 1 of arXiv:1906.06306) is
 *   B1 = B - (c/2) curl+ E                     (Eq. fdB, half step)
 *   e, b = interp(E, B1; x); u' = Boris(u, e, b)          (App. C)
 *   x' = x + c u'/gamma(u');  J = sum ZigZag(x, x')        (Eq. fdX, App. D)
 *   B2 = B1 - (c/2) curl+ E
 *   E' = E + c curl- B2 - F^p J                 (Eq. fdE, add_cur, Binomial2)
 * and the adjoint runs it backwards.  On a periodic lattice the forward
 * difference's transpose is minus the backward one, so (curl+)^T = curl- and
 * (curl-)^T = curl+; the Binomial2 filter is symmetric.  Every other piece is
 * the chain rule through the formulas the forward step uses (the floor of a
 * position and the branch of the ZigZag relay point are locally constant). */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "pic_oracle.h"

enum { EX, EY, EZ, BX, BY, BZ, JX, JY, JZ };

static long wrapa(long i, long n) {
  long r = i % n;
  return r < 0 ? r + n : r;
}

static long ncells(const orc_grid* g) { return (long)g->nx * g->ny * g->nz; }

static long idx(const orc_grid* g, long i, long j, long k) {
  return (wrapa(k, g->nz) * g->ny + wrapa(j, g->ny)) * g->nx + wrapa(i, g->nx);
}

static double ext(const orc_grid* g, int d) { return d == 0 ? g->nx : d == 1 ? g->ny : g->nz; }

/* Difference of plane `comp` along axis d at (i,j,k): forward (A(p+e_d) -
 * A(p)) or backward (A(p) - A(p-e_d)); zero along a non-gridded axis. */
static double diff(const orc_grid* g, const double* A, int comp, int d, int fwd, long i, long j,
                   long k) {
  if (d >= g->dim) return 0.0;
  const long P = ncells(g);
  const long di = d == 0, dj = d == 1, dk = d == 2;
  if (fwd) return A[comp * P + idx(g, i + di, j + dj, k + dk)] - A[comp * P + idx(g, i, j, k)];
  return A[comp * P + idx(g, i, j, k)] - A[comp * P + idx(g, i - di, j - dj, k - dk)];
}

/* out[0..2] += s * curl(A[src..src+2]) at every point, forward or backward
 * differences. */
static void add_curl(const orc_grid* g, const double* A, int src, int fwd, double s, double* out) {
  const long P = ncells(g);
  for (long k = 0; k < g->nz; ++k)
    for (long j = 0; j < g->ny; ++j)
      for (long i = 0; i < g->nx; ++i) {
        const long p = idx(g, i, j, k);
        const double cx = diff(g, A, src + 2, 1, fwd, i, j, k) - diff(g, A, src + 1, 2, fwd, i, j, k);
        const double cy = diff(g, A, src + 0, 2, fwd, i, j, k) - diff(g, A, src + 2, 0, fwd, i, j, k);
        const double cz = diff(g, A, src + 1, 0, fwd, i, j, k) - diff(g, A, src + 0, 1, fwd, i, j, k);
        out[0 * P + p] += s * cx;
        out[1 * P + p] += s * cy;
        out[2 * P + p] += s * cz;
      }
}

void orc_adj_push_half_b(const orc_grid* g, double* A) {
  /* forward B -= (c/2) curl+ E  ->  Ebar -= (c/2) curl- Bbar */
  const long P = ncells(g);
  double* d = (double*)calloc(3 * (size_t)P, sizeof(double));
  add_curl(g, A, BX, 0, -0.5 * g->c, d);
  for (long p = 0; p < 3 * P; ++p) A[EX * P + p] += d[p];
  free(d);
}

void orc_adj_push_e(const orc_grid* g, double* A) {
  /* forward E += c curl- B - J  ->  Bbar += c curl+ Ebar, Jbar = -Ebar */
  const long P = ncells(g);
  double* d = (double*)calloc(3 * (size_t)P, sizeof(double));
  add_curl(g, A, EX, 1, g->c, d);
  for (long p = 0; p < 3 * P; ++p) {
    A[BX * P + p] += d[p];
    A[JX * P + p] = -A[EX * P + p];
  }
  free(d);
}

/* Staggered position of each field component inside its cell (Sect. 2.3.1). */
static const double STAGA[6][3] = {
    {0.5, 0.0, 0.0}, {0.0, 0.5, 0.0}, {0.0, 0.0, 0.5},
    {0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}, {0.5, 0.5, 0.0},
};

/* Linear weight of corner o (bits per axis) and its derivative along axis d. */
static double corner_weight(const orc_grid* g, const double* w, const int* o, int skip_axis,
                            int dd) {
  double wt = 1.0;
  for (int d = 0; d < g->dim; ++d) {
    if (d == skip_axis) continue;
    if (d == dd)
      wt *= o[d] ? 1.0 : -1.0;
    else
      wt *= o[d] ? w[d] : 1.0 - w[d];
  }
  return wt;
}

/* Gather of component comp at x (the forward LinearInterpolator) and, with
 * vbar != 0, its reverse: A[comp] += weights * vbar, xbar += d(value)/dx * vbar. */
static double gather1(const orc_grid* g, const double* F, int comp, const double* x, double vbar,
                      double* A, double* xbar) {
  const long P = ncells(g);
  long i0[3] = {0, 0, 0};
  double w[3] = {0.0, 0.0, 0.0};
  for (int d = 0; d < g->dim; ++d) {
    const double xi = x[d] - STAGA[comp][d];
    i0[d] = (long)floor(xi);
    w[d] = xi - (double)i0[d];
  }
  double s = 0.0;
  const int nc = 1 << g->dim;
  for (int c = 0; c < nc; ++c) {
    const int o[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
    const long p = idx(g, i0[0] + o[0], i0[1] + o[1], i0[2] + o[2]);
    const double f = F[comp * P + p];
    s += corner_weight(g, w, o, -1, -1) * f;
    if (A) {
      A[comp * P + p] += corner_weight(g, w, o, -1, -1) * vbar;
      for (int d = 0; d < g->dim; ++d) xbar[d] += corner_weight(g, w, o, -1, d) * f * vbar;
    }
  }
  return s;
}

static void crossa(const double* a, const double* b, double* r) {
  r[0] = a[1] * b[2] - a[2] * b[1];
  r[1] = a[2] * b[0] - a[0] * b[2];
  r[2] = a[0] * b[1] - a[1] * b[0];
}

/* Boris (App. C) forward and reverse: u' = u3/c with u1 = c u + hs e,
 * g1 = (1 + u1^2/c^2)^(-1/2), t = (hs/c) g1 b, f = 2/(1 + t^2),
 * v = f (u1 + u1 x t), u3 = u1 + v x t + hs e.  Given up_bar (gradient of u'),
 * writes u_bar, e_bar, b_bar. */
static void boris_adj(const double* u, const double* e, const double* b, double qm, double c,
                      const double* up_bar, double* u_bar, double* e_bar, double* b_bar) {
  const double hs = 0.5 * qm;
  double u1[3], t[3], s[3], v[3], x1[3];
  for (int a = 0; a < 3; ++a) u1[a] = c * u[a] + hs * e[a];
  const double g1 = 1.0 / sqrt(1.0 + (u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]) / (c * c));
  const double tf = hs / c * g1;
  for (int a = 0; a < 3; ++a) t[a] = tf * b[a];
  const double den = 1.0 + t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
  const double f = 2.0 / den;
  crossa(u1, t, x1);
  for (int a = 0; a < 3; ++a) {
    s[a] = u1[a] + x1[a];
    v[a] = f * s[a];
  }
  /* reverse */
  double u3b[3], u1b[3], vb[3], tb[3] = {0, 0, 0}, sb[3], tmp[3];
  for (int a = 0; a < 3; ++a) {
    u3b[a] = up_bar[a] / c;
    u1b[a] = u3b[a];
    e_bar[a] = hs * u3b[a];
  }
  /* w = v x t: vbar = t x wbar, tbar += wbar x v */
  crossa(t, u3b, vb);
  crossa(u3b, v, tmp);
  for (int a = 0; a < 3; ++a) tb[a] += tmp[a];
  /* v = f s */
  double fb = 0.0;
  for (int a = 0; a < 3; ++a) {
    fb += vb[a] * s[a];
    sb[a] = f * vb[a];
  }
  /* s = u1 + u1 x t: u1bar += sbar + t x sbar, tbar += sbar x u1 */
  crossa(t, sb, tmp);
  for (int a = 0; a < 3; ++a) u1b[a] += sb[a] + tmp[a];
  crossa(sb, u1, tmp);
  for (int a = 0; a < 3; ++a) tb[a] += tmp[a];
  /* f = 2/den: denbar = -f^2/2 fbar; den = 1 + t.t */
  const double denb = -0.5 * f * f * fb;
  for (int a = 0; a < 3; ++a) tb[a] += 2.0 * t[a] * denb;
  /* t = tf b */
  double tfb = 0.0;
  for (int a = 0; a < 3; ++a) {
    tfb += tb[a] * b[a];
    b_bar[a] = tf * tb[a];
  }
  /* tf = (hs/c) g1; g1 = (1 + u1^2/c^2)^(-1/2): dg1/du1 = -g1^3 u1 / c^2 */
  const double g1b = tfb * hs / c;
  for (int a = 0; a < 3; ++a) u1b[a] += -g1b * g1 * g1 * g1 * u1[a] / (c * c);
  /* u1 = c u + hs e */
  for (int a = 0; a < 3; ++a) {
    u_bar[a] = c * u1b[a];
    e_bar[a] += hs * u1b[a];
  }
}

/* Reverse of one ZigZag segment's deposit (the oracle's deposit_segment):
 * from Jbar at the words of cell I, accumulate Dbar (segment displacement)
 * and Wbar (segment weights). */
static void segment_adj(const orc_grid* g, const double* A, const long* I, double q,
                        const double* Ds, const double* W, double* Dbar, double* Wbar) {
  const long P = ncells(g);
  for (int a = 0; a < 3; ++a) {
    const double Fl = q * Ds[a];
    for (int c = 0; c < 8; ++c) {
      const int o[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
      int skip = 0;
      for (int d = 0; d < 3; ++d)
        if ((d >= g->dim || d == a) && o[d]) skip = 1;
      if (skip) continue;
      const double jb = A[(JX + a) * P + idx(g, I[0] + o[0], I[1] + o[1], I[2] + o[2])];
      double wt = corner_weight(g, W, o, a, -1);
      double sgn = 0.0;
      int bb = 0, cc = 0;
      if (g->dim == 3) {
        bb = (a + 1) % 3;
        cc = (a + 2) % 3;
        sgn = o[bb] == o[cc] ? 1.0 : -1.0;
        wt += sgn * Ds[bb] * Ds[cc] / 12.0;
      }
      Dbar[a] += q * wt * jb;
      for (int d = 0; d < g->dim; ++d)
        if (d != a) Wbar[d] += Fl * jb * corner_weight(g, W, o, a, d);
      if (g->dim == 3) {
        Dbar[bb] += Fl * jb * sgn * Ds[cc] / 12.0;
        Dbar[cc] += Fl * jb * sgn * Ds[bb] / 12.0;
      }
    }
  }
}

/* Reverse of the ZigZag current of a move x1 -> x2 = x1 + dn (gridded rows of
 * x1, x2; dn on every axis): x1bar, x2bar on gridded axes, dnbar on the
 * others. */
static void zigzag_adj(const orc_grid* g, const double* A, const double* x1, const double* x2,
                       const double* dn, double q, double* x1b, double* x2b, double* dnb) {
  long i1[3] = {0, 0, 0}, i2[3] = {0, 0, 0};
  double xr[3], D1[3], D2[3], W1[3] = {0, 0, 0}, W2[3] = {0, 0, 0};
  int mid[3] = {0, 0, 0};
  for (int d = 0; d < 3; ++d) {
    if (d < g->dim) {
      i1[d] = (long)floor(x1[d]);
      i2[d] = (long)floor(x2[d]);
      const double lo = (double)(i1[d] < i2[d] ? i1[d] : i2[d]) + 1.0;
      const double hi = (double)(i1[d] > i2[d] ? i1[d] : i2[d]);
      const double m = 0.5 * (x1[d] + x2[d]);
      xr[d] = fmin(lo, fmax(hi, m));
      mid[d] = m > hi && m < lo;
      W1[d] = 0.5 * (x1[d] + xr[d]) - (double)i1[d];
      W2[d] = 0.5 * (x2[d] + xr[d]) - (double)i2[d];
      D1[d] = xr[d] - x1[d];
      D2[d] = x2[d] - xr[d];
    } else {
      D1[d] = D2[d] = 0.5 * dn[d];
    }
  }
  double D1b[3] = {0, 0, 0}, D2b[3] = {0, 0, 0}, W1b[3] = {0, 0, 0}, W2b[3] = {0, 0, 0};
  segment_adj(g, A, i1, q, D1, W1, D1b, W1b);
  segment_adj(g, A, i2, q, D2, W2, D2b, W2b);
  for (int d = 0; d < 3; ++d) {
    if (d < g->dim) {
      const double xrb = D1b[d] - D2b[d] + 0.5 * (W1b[d] + W2b[d]);
      x1b[d] = -D1b[d] + 0.5 * W1b[d];
      x2b[d] = D2b[d] + 0.5 * W2b[d];
      if (mid[d]) {
        x1b[d] += 0.5 * xrb;
        x2b[d] += 0.5 * xrb;
      }
      dnb[d] = 0.0;
    } else {
      x1b[d] = x2b[d] = 0.0;
      dnb[d] = 0.5 * (D1b[d] + D2b[d]);
    }
  }
}

void orc_adj_particles(const orc_grid* g, const double* F1, const double* x, const double* u,
                       long n, double q, double qm, double* xbar, double* ubar, double* A) {
  const double c = g->c;
  for (long p = 0; p < n; ++p) {
    double xp[3] = {0, 0, 0}, up[3], e[3], b[3];
    for (int d = 0; d < g->dim; ++d) xp[d] = x[d * n + p];
    for (int a = 0; a < 3; ++a) up[a] = u[a * n + p];
    for (int a = 0; a < 3; ++a) {
      e[a] = gather1(g, F1, EX + a, xp, 0.0, NULL, NULL);
      b[a] = gather1(g, F1, BX + a, xp, 0.0, NULL, NULL);
    }
    double u2[3] = {up[0], up[1], up[2]};
    orc_boris(u2, e, b, qm, c);
    const double gam = sqrt(1.0 + u2[0] * u2[0] + u2[1] * u2[1] + u2[2] * u2[2]);
    double dn[3], x2[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a) dn[a] = c * u2[a] / gam;
    for (int d = 0; d < g->dim; ++d) x2[d] = xp[d] + dn[d];
    /* reverse: x' = wrap(x + dn) */
    double xb[3] = {0, 0, 0}, dnb[3] = {0, 0, 0}, u2b[3];
    for (int d = 0; d < g->dim; ++d) {
      xb[d] = xbar[d * n + p];
      dnb[d] = xbar[d * n + p];
    }
    for (int a = 0; a < 3; ++a) u2b[a] = ubar[a * n + p];
    /* ZigZag J(x, x + dn) */
    double zx1[3], zx2[3], zdn[3];
    zigzag_adj(g, A, xp, x2, dn, q, zx1, zx2, zdn);
    for (int d = 0; d < 3; ++d) {
      if (d < g->dim) {
        xb[d] += zx1[d] + zx2[d];
        dnb[d] += zx2[d];
      } else {
        dnb[d] += zdn[d];
      }
    }
    /* dn = c u2 / gamma: u2bar += (c/gamma) (dnbar - u2 (u2.dnbar) / gamma^2) */
    const double ud = u2[0] * dnb[0] + u2[1] * dnb[1] + u2[2] * dnb[2];
    for (int a = 0; a < 3; ++a) u2b[a] += c / gam * (dnb[a] - u2[a] * ud / (gam * gam));
    double ub[3], eb[3], bb[3];
    boris_adj(up, e, b, qm, c, u2b, ub, eb, bb);
    for (int a = 0; a < 3; ++a) {
      gather1(g, F1, EX + a, xp, eb[a], A, xb);
      gather1(g, F1, BX + a, xp, bb[a], A, xb);
    }
    for (int d = 0; d < g->dim; ++d) xbar[d * n + p] = xb[d];
    for (int a = 0; a < 3; ++a) ubar[a * n + p] = ub[a];
  }
}

void orc_adj_step(const orc_grid* g, const double* F, double** x, double** u, const long* n,
                  const double* q, const double* m, int ns, int passes, double** xbar,
                  double** ubar, double* A, double* work) {
  const long P = ncells(g);
  /* forward fields seen by the particles: E^n and B1 = B - (c/2) curl+ E */
  memcpy(work, F, sizeof(double) * 9 * (size_t)P);
  orc_push_half_b(g, work);
  orc_adj_push_e(g, A);                 /* E' = E + c curl- B2 - Jf */
  orc_filter_binomial(g, A, passes);    /* Jf = F^p J (symmetric) */
  orc_adj_push_half_b(g, A);            /* B2 = B1 - (c/2) curl+ E */
  for (int s = 0; s < ns; ++s)          /* gather, Boris, move, ZigZag */
    orc_adj_particles(g, work, x[s], u[s], n[s], q[s], q[s] / m[s], xbar[s], ubar[s], A);
  orc_adj_push_half_b(g, A);            /* B1 = B - (c/2) curl+ E */
  for (long p = 0; p < 3 * P; ++p) A[JX * P + p] = 0.0;
}
