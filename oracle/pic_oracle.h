/* FP64 CPU oracle of the relativistic PIC time step of the Runko paper
 * (Nattila, arXiv:1906.06306).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously correct
 * reference that the CUDA path is checked against.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it; the product
 * library never links, calls or falls back to it, and it shares no code,
 * header, table or helper with the CUDA path.
 *
 * Conventions (Sect. 2.3, Appendix A): code units with dx = dt = 1; the
 * Courant number c is the only constant in the field equations.
 *
 * Fields: double[9][nz][ny][nx], planes Ex Ey Ez Bx By Bz Jx Jy Jz.  Plane
 * element [i,j,k] lives at the Yee point of Sect. 2.3.1:
 *   Ex (i+1/2, j, k)   Ey (i, j+1/2, k)   Ez (i, j, k+1/2)
 *   Bx (i, j+1/2, k+1/2)   By (i+1/2, j, k+1/2)   Bz (i+1/2, j+1/2, k)
 *   J shares the points of E; charge density lives on the nodes (i, j, k).
 * In D < 3 the missing dimensions are not
 * gridded: nothing varies along them and they have extent 1.
 *
 * Particles: double x[3][n] (absolute positions, only the first D rows are
 * used, each in [0, n_d)), double u[3][n] (four-velocity in units of c).
 * All boundaries are periodic unless the shock boundaries are set (a wall
 * and an injector along x, orc_set_wall / orc_inject).
 */
#ifndef PIC_ORACLE_H
#define PIC_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int dim;        /* 1, 2 or 3 gridded dimensions */
  int nx, ny, nz; /* cells per dimension (1 for non-gridded ones) */
  double c;       /* Courant number */
} orc_grid;

/* Field solver, Eq. (fdB) over half a step: B -= (c/2) curl E. */
void orc_push_half_b(const orc_grid* g, double* F);
/* Spatial order of orc_push_half_b / orc_push_e: 2 (FDTD2, default) or 4
 * (FDTD4: fourth-order staggered differences, coefficients 9/8 and -1/24). */
void orc_set_field_order(int order);
/* Field solver, curl part of Eq. (fdE): E += c curl B. */
void orc_push_e(const orc_grid* g, double* F);
/* add_cur of Table 1, current part of Eq. (fdE): E -= J. */
void orc_add_cur(const orc_grid* g, double* F);
/* Binomial2 filter (Table 2): `passes` passes of (1/4, 1/2, 1/4) along every
 * gridded dimension on Jx, Jy, Jz. */
void orc_filter_binomial(const orc_grid* g, double* F, int passes);

/* LinearInterpolator: E and B at position x (3 values, only the gridded ones
 * are read) by first-order weighting of each staggered component. */
void orc_interp(const orc_grid* g, const double* F, const double* x, double* e, double* b);
/* Relativistic Boris scheme of Appendix C, u (units of c) advanced in place by
 * one step; qm = q/m of the species (s-hat). */
void orc_boris(double* u, const double* e, const double* b, double qm, double c);
/* Higuera-Cary pusher (Table 2, HigueraCaryPusher; Higuera and Cary 2017), the
 * alternative the paper uses for its shock run: the Boris steps with the
 * rotation's Lorentz factor taken from the quadratic that makes the E x B drift
 * exact.  Same arguments and units as orc_boris. */
void orc_higuera_cary(double* u, const double* e, const double* b, double qm, double c);
/* Pusher selection for orc_push_particles / orc_step: 0 Boris, 1 Higuera-Cary. */
void orc_set_pusher(int pusher);

/* ZigZag current of Appendix D for one particle moving from x1 to x2
 * (unwrapped: x2 - x1 is the displacement; rows of non-gridded dimensions
 * carry only the displacement), charge q, added into the J planes of F. */
void orc_zigzag(const orc_grid* g, double* F, const double* x1, const double* x2, double q);

/* interp_em + push of Table 1 for every particle of a species: gather, Boris,
 * position update of Eq. (fdX) with periodic wrap.  The pre-move positions are
 * written to x_old[3][n] (rows of non-gridded dims are 0) and the
 * displacements to dx[3][n], both consumed by orc_deposit. */
void orc_push_particles(const orc_grid* g, const double* F, double* x, double* u, long n,
                        double qm, double* x_old, double* dx);
/* comp_curr of Table 1 for one species: ZigZag from x_old to x_old + dx. */
void orc_deposit(const orc_grid* g, double* F, const double* x_old, const double* dx, long n,
                 double q);
/* The same ZigZag deposit adding |term| for each of Appendix D's terms: per
 * current word the sum of the magnitudes of its contributions. */
void orc_deposit_abs(const orc_grid* g, double* F, const double* x_old, const double* dx, long n,
                     double q);

/* Shock boundaries (Sect. 4.2).  orc_set_wall(w, i_zero) with w >= 1 puts a
 * conducting wall on the node plane x = w for orc_push_particles, orc_deposit
 * and orc_step (w = 0: none): particles that cross it are reflected
 * specularly and their current follows the reflected path; after each field
 * update orc_step applies orc_wall_fields. */
void orc_set_wall(long w, long i_zero);
/* Mirror-image field boundary of a perfect conductor at the node x = w, and
 * zero E and B at i >= i_zero. */
void orc_wall_fields(const orc_grid* g, double* F, long w, long i_zero);
/* Receding injector: the particles of an upstream template (xt[3][nt] in
 * [0, lt) x ny x nz sorted by x, ut[3][nt]) that cross the injector
 * X(s) = min(x0 + v_inj s, x_max) during step s, the template moving at -v_up;
 * written to xo[3][cap], uo[3][cap]; returns the count or -1 (cap too small). */
long orc_inject(const double* xt, const double* ut, long nt, long lt, double x0, double x_max,
                double v_inj, double v_up, long s, double* xo, double* uo, long cap);

/* One full time step in the order of Table 1 for `ns` species:
 * B half, interp_em + push (all species), B half, push_e, clear J and
 * comp_curr (all species), `passes` Binomial2 passes, add_cur.
 * x[s], u[s] point to each species' arrays; work must hold 6 * sum(n) doubles. */
void orc_step(const orc_grid* g, double* F, double** x, double** u, const long* n,
              const double* q, const double* m, int ns, int passes, double* work);

/* Reverse mode (discrete adjoint) of orc_step, FDTD2 and Boris only
 * (pic_oracle_adj.c).  A holds adjoint field planes in the field layout
 * (Ebar, Bbar; the J planes are scratch): on entry the gradient of a loss
 * with respect to E and B after the step, on exit with respect to E and B
 * before it.  xbar[s] (gridded rows of float[3][n]) and ubar[s] likewise for
 * the particles.  F, x, u: the forward state at the start of the step.  work
 * must hold 9 * ncells doubles. */
void orc_adj_step(const orc_grid* g, const double* F, double** x, double** u, const long* n,
                  const double* q, const double* m, int ns, int passes, double** xbar,
                  double** ubar, double* A, double* work);
/* Pieces of orc_adj_step: adjoints of orc_push_half_b, of orc_push_e with
 * orc_add_cur (Jbar = -Ebar), and of the particle part (F1 = E and the B of
 * the first half step). */
void orc_adj_push_half_b(const orc_grid* g, double* A);
void orc_adj_push_e(const orc_grid* g, double* A);
void orc_adj_particles(const orc_grid* g, const double* F1, const double* x, const double* u,
                       long n, double q, double qm, double* xbar, double* ubar, double* A);

/* Charge density on the nodes, first-order (cloud-in-cell) shape, added into
 * rho[nz][ny][nx]. */
void orc_charge_density(const orc_grid* g, const double* x, long n, double q, double* rho);
/* Discrete divergence of E on the nodes (backward differences), written to div. */
void orc_div_e(const orc_grid* g, const double* F, double* div);
/* Discrete divergence of B at the cell centres (forward differences). */
void orc_div_b(const orc_grid* g, const double* F, double* div);
/* Field energies 0.5 sum E^2 and 0.5 sum B^2 (out[0], out[1]). */
void orc_field_energy(const orc_grid* g, const double* F, double* out);
/* Kinetic energy sum m c^2 (gamma - 1) of one species. */
double orc_kinetic_energy(const double* u, long n, double m, double c);

#ifdef __cplusplus
}
#endif
#endif
