"""Pins of the oracle's shock boundaries (Sect. 4.2): the conducting wall
(specular reflection, charge continuity of reflected particles, the standing
waves of a perfect conductor, Gauss law) and the receding injector (the box
fills with the advected upstream template: no gap, no duplicate, right time).
No CUDA code is involved."""
import math

import numpy as np
import pytest

import workloads

C = 0.45


@pytest.fixture
def wall(orc):
    """Set the oracle's wall for one test and always clear it afterwards."""
    def set_(w, i_zero):
        orc.set_wall(w, i_zero)
    yield set_
    orc.set_wall(0, 0)


def _rho(orc, g, x, q):
    return sum(orc.charge_density(g, [orc.Species(q[p], 1.0, x[:, p:p + 1], np.zeros((3, 1)))])
               for p in range(x.shape[1]))


def _div_j(orc, g, F):
    G = g.zeros()
    G[0:3] = F[6:9]
    return orc.div_e(g, G)


def test_wall_reflects_specularly(orc, wall):
    """Zero fields: a particle heading into the wall at x = w ends at the
    mirror image 2 w - x of its free-flight position, with u_x reversed and
    |u| kept; the other coordinates advance freely."""
    g = orc.Grid(2, 16, 8, 1, C)
    w = 3
    wall(w, 14)
    F = g.zeros()
    u0 = np.array([-3.0, 1.0, 0.5])
    x0 = np.array([w + 0.2, 5.3, 0.0])
    sp = orc.Species(-1.0, 1.0, x0.reshape(3, 1).copy(), u0.reshape(3, 1).copy())
    orc.push_particles(g, F, sp)
    gam = math.sqrt(1.0 + (u0 ** 2).sum())
    free = x0 + C * u0 / gam
    assert free[0] < w  # the move does cross the wall
    assert sp.x[0, 0] == pytest.approx(2 * w - free[0], abs=1e-14)
    assert sp.x[1, 0] == pytest.approx(free[1], abs=1e-14)
    assert sp.u[:, 0] == pytest.approx([3.0, 1.0, 0.5], abs=0.0)


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_reflected_current_conserves_charge(orc, wall, dim):
    """rho(after) - rho(before) + div^- J = 0 on every node, the wall node
    included, when many particles near the wall are pushed into it: the
    current follows the reflected path (Appendix B's continuity)."""
    nx, ny, nz = (12, 5, 4)[:dim] + (1,) * (3 - dim)
    g = orc.Grid(dim, nx, ny, nz, C)
    w = 2
    wall(w, nx - 1)
    rs = np.random.default_rng(31)
    n = 300
    x = np.zeros((3, n))
    x[0] = w + rs.uniform(0.0, 0.44, n)
    for d in range(1, dim):
        x[d] = rs.uniform(0.0, (ny, nz)[d - 1], n)
    u = rs.normal(0.0, 2.0, (3, n))
    u[0] = -np.abs(u[0]) - 0.5
    q = rs.choice([-1.3, 0.7], n)
    F = g.zeros()
    rho0 = _rho(orc, g, x, q)
    sps = [orc.Species(q[p], 1.0, x[:, p:p + 1].copy(), u[:, p:p + 1].copy()) for p in range(n)]
    crossed = 0
    for sp in sps:
        x_old, dx = orc.push_particles(g, F, sp)
        crossed += int(x_old[0, 0] + dx[0, 0] < w)
        orc.deposit(g, F, x_old, dx, sp.q)
    assert crossed > n // 4
    x1 = np.concatenate([sp.x for sp in sps], axis=1)
    assert x1[0].min() >= w
    res = _rho(orc, g, x1, q) - rho0 + _div_j(orc, g, F)
    assert np.abs(res).max() < 1e-12


@pytest.mark.parametrize("pol", ["ey_bz", "ez_by"])
@pytest.mark.parametrize("dim", [1, 2])
def test_conducting_wall_standing_wave(orc, wall, pol, dim):
    """A vacuum standing wave E_t = sin(k (x - w)) cos(w t) with its B partner
    is an exact discrete solution of FDTD2 when the wall sits at its node
    (tangential E odd about the wall, tangential B even), with
    sin(omega/2) = c sin(k/2).  The oracle keeps it to round-off wherever the
    zeroed region beyond i_zero cannot reach (one cell per step)."""
    nx = 64
    g = orc.Grid(dim, nx, 4, 1, C)
    w, i_zero, nsteps = 5, 58, 20
    wall(w, i_zero)
    k = 0.37
    om = 2.0 * math.asin(C * math.sin(k / 2.0))
    xi = np.arange(nx, dtype=np.float64)

    def fields(n):
        F = g.zeros()
        e = np.sin(k * (xi - w)) * math.cos(om * n)
        b = np.cos(k * (xi + 0.5 - w)) * math.sin(om * (n - 0.5))
        if pol == "ey_bz":
            F[1] = e
            F[5] = -b
        else:
            F[2] = e
            F[4] = b
        return F

    F = fields(0)
    orc.wall_fields(g, F, w, i_zero)
    F[:, :, :, i_zero:] = 0.0
    ref0 = fields(0)
    ok = slice(0, i_zero - 1)
    assert np.abs(F[:, :, :, ok] - ref0[:, :, :, ok]).max() < 1e-14
    for _ in range(nsteps):
        orc.step(g, F, [])
    ref = fields(nsteps)
    ok = slice(0, i_zero - nsteps - 2)
    assert np.abs(F[:, :, :, ok] - ref[:, :, :, ok]).max() < 1e-12
    assert np.abs(ref[:, :, :, ok]).max() > 0.5


def _tube(dim, **kw):
    args = dict(dim=dim, nx=48, ny=6, nz=4, ppc=3, gamma_flow=3.0, theta=0.05, r_p=3.0,
                wall=3, x_inj=20, x_max=40.0, lt=8, filter_passes=0, seed=77)
    args.update(kw)
    return workloads.shock_tube(**args)


@pytest.mark.parametrize("dim,passes", [(2, 0), (2, 2), (3, 1)])
def test_shock_tube_gauss_law(orc, wall, dim, passes):
    """Wall, injector and a warm counter-streaming plasma: div E - F^p(rho) stays
    at round-off on every node between the wall and the zeroed region (the
    wall node itself carries the conductor's surface charge), while charge
    separation makes div E large."""
    pl = _tube(dim, filter_passes=passes)
    g, F, sp = orc.from_plasma(pl)
    w, i_zero, inj = orc.shock_from_plasma(pl)
    wall(w, i_zero)
    orc.step_shock(g, F, sp, inj, 0, passes=passes, nsteps=40)
    assert sp[0].n > pl.species[0].n  # the injector let particles in
    assert min(s.x[0].min() for s in sp) >= w
    res = orc.gauss_residual(g, F, sp, passes)
    inner = res[..., w + 1:i_zero]
    scale = np.abs(orc.div_e(g, F)[..., w + 1:i_zero]).max()
    assert scale > 1e-5
    assert np.abs(inner).max() < 1e-12 * max(1.0, scale / 1e-3)
    # a perfect conductor: tangential E vanishes on the wall plane although
    # reflected particles leave tangential current on the wall node
    assert np.abs(F[1:3, ..., w]).max() == 0.0
    assert np.abs(F[7, ..., w]).max() > 0.0


@pytest.mark.parametrize("x_max", [40.0, 27.5])
def test_injector_fills_the_box_with_the_advected_template(orc, wall, x_max):
    """No fields, no wall, a cold template moving at exactly -v_up: after s
    steps the particles are exactly the template copies m >= 0 advected to
    x_t + m lt + x0 - v_up s that lie behind the injector (template coordinate
    below (X(s) - x0) + v_up s), each once, also after the injector stops at
    x_max."""
    dim, lt, x0, nx, ny = 2, 8, 20.0, 48, 6
    g = orc.Grid(dim, nx, ny, 1, C)
    rs = np.random.default_rng(5)
    nt = 40
    xt = np.zeros((3, nt))
    xt[0] = np.sort(rs.uniform(0.0, lt, nt).astype(np.float32).astype(np.float64))
    xt[1] = rs.uniform(0.0, ny, nt).astype(np.float32)
    ut = np.zeros((3, nt))
    ut[0] = -2.0
    v_up = -C * ut[0, 0] / math.sqrt(1.0 + ut[0, 0] ** 2)
    inj = orc.Injector([(xt, ut)], lt, x0, x_max, C, v_up)
    # a vanishing charge: the particles' own field must not deflect them
    sp = [orc.Species(-1e-12, 1.0, np.zeros((3, 0)), np.zeros((3, 0)))]
    F = g.zeros()
    steps = 30
    orc.step_shock(g, F, sp, inj, 0, nsteps=steps)
    front = (min(x0 + C * steps, x_max) - x0) + v_up * steps
    exp = []
    for m in range(int(front // lt) + 1):
        for k in range(nt):
            if xt[0, k] + m * lt < front:
                exp.append((xt[0, k] + m * lt + x0 - v_up * steps, xt[1, k]))
    exp = np.array(sorted(exp))
    got = np.array(sorted(zip(sp[0].x[0], sp[0].x[1])))
    assert got.shape == exp.shape and len(exp) > 2 * nt
    assert np.abs(got - exp).max() < 1e-6
    assert np.all(got[:, 0] < min(x0 + C * steps, x_max))


def test_injected_pairs_are_co_located(orc, wall):
    pl = _tube(2)
    g, F, sp = orc.from_plasma(pl)
    w, i_zero, inj = orc.shock_from_plasma(pl)
    wall(w, i_zero)
    n0 = sp[0].n
    counts = inj.inject(0, sp)
    assert counts[0] == counts[1] > 0
    assert np.array_equal(sp[0].x[:, n0:], sp[1].x[:, n0:])


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_reflected_deposit_equals_the_integral_along_the_true_path(orc, wall, dim):
    """Brute force: the current of a reflected particle equals the sum of the
    ZigZag currents of many short straight moves along its true trajectory
    (free flight to the wall plane, mirrored afterwards).  Inside one cell the
    ZigZag current of a straight move is the exact line integral of the
    first-order weights, so the sum is additive and the two must agree to
    round-off; a misplaced crossing point or a missing segment does not.
    The exception is Jz in 2D: not gridded, weighted by two gridded weights at
    each half's midpoint, which is not the line integral of their product, so
    only its lattice sum q dz is compared."""
    nx, ny, nz = (10, 6, 5)[:dim] + (1,) * (3 - dim)
    g = orc.Grid(dim, nx, ny, nz, C)
    w = 2
    wall(w, nx - 1)
    rs = np.random.default_rng(41 + dim)
    for trial in range(20):
        x1 = np.zeros(3)
        x1[0] = w + rs.uniform(0.02, 0.4)
        for d in range(1, dim):
            x1[d] = rs.integers(0, (ny, nz)[d - 1]) + rs.uniform(0.3, 0.7)
        u = np.array([-rs.uniform(1.0, 6.0), rs.normal(0, 0.3), rs.normal(0, 0.3)])
        q = rs.choice([-1.0, 0.6])
        dx = C * u / math.sqrt(1.0 + (u ** 2).sum())
        if x1[0] + dx[0] >= w:
            continue
        F = g.zeros()
        orc.deposit(g, F, x1.reshape(3, 1), dx.reshape(3, 1), q)
        t_c = (x1[0] - w) / (-dx[0])  # fraction of the step spent before the wall

        def path(t):
            p = x1 + t * dx
            if t > t_c:
                p[0] = 2 * w - p[0]
            return p

        ts = sorted(set(np.linspace(0.0, 1.0, 65).tolist() + [t_c]))
        G = g.zeros()
        for a, b in zip(ts[:-1], ts[1:]):
            pa, pb = path(a), path(b)
            if b == t_c:
                pb[0] = w
            if a == t_c:
                pa[0] = w
            orc.zigzag(g, G, pa, pb, q)
        comps = [6, 7] if dim == 2 else [6, 7, 8]
        assert np.abs(F[comps] - G[comps]).max() < 1e-13
        assert F[8].sum() == pytest.approx(q * dx[2], abs=1e-14)
