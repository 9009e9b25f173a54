"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms
(Boris rotation angle, pure-E kick, E x B drift, the Yee dispersion relation,
the binomial filter's Fourier response and impulse response), exact
reproduction properties (linear interpolation of linear fields), hand sums
(tests/golden/zigzag_hand_sums.json, Appendix D) and invariants (discrete
continuity and Gauss law of Appendix B, div B = 0, Weibel growth rate of
Sect. 4.1).  No CUDA code is involved.
"""
import json
import math
import os

import numpy as np
import pytest

C = 0.45
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# Sect. 2.3.1: position of each component inside its cell (x, y, z)
E_STAG = [(0.5, 0, 0), (0, 0.5, 0), (0, 0, 0.5)]
B_STAG = [(0, 0.5, 0.5), (0.5, 0, 0.5), (0.5, 0.5, 0)]


# ----------------------------------------------------------------- Boris ----

@pytest.mark.parametrize("qm", [1.0, -1.0, 0.5])
@pytest.mark.parametrize("bz", [0.05, 0.3, 2.0])
def test_boris_uniform_b_rotation_closed_form(orc, qm, bz):
    """E = 0, uniform B along z: each Boris step is an exact rotation about z by
    2 atan(|t|), t = s B / (2 c gamma), clockwise for s B > 0 (the v x B force
    of a positive charge moving along +x points to -y); |u| is conserved."""
    u0 = np.array([1.7, -0.6, 0.4])
    gam = math.sqrt(1.0 + u0 @ u0)
    ang = 2.0 * math.atan(qm * bz / (2.0 * C * gam))
    u = u0.copy()
    nsteps = 500
    for _ in range(nsteps):
        u = orc.boris(u, [0, 0, 0], [0, 0, bz], qm, C)
    a = nsteps * ang
    expect = np.array([u0[0] * math.cos(a) + u0[1] * math.sin(a),
                       -u0[0] * math.sin(a) + u0[1] * math.cos(a), u0[2]])
    assert np.allclose(u, expect, rtol=0, atol=1e-10)
    assert abs(np.linalg.norm(u) - np.linalg.norm(u0)) < 1e-12


def test_boris_pure_e_kick_exact(orc):
    """B = 0: the two half kicks add to u_new = u + s E / c exactly."""
    u0 = np.array([0.3, -0.2, 0.1])
    e = np.array([0.01, -0.02, 0.03])
    for qm in (1.0, -1.0, 0.25):
        u = orc.boris(u0, e, [0, 0, 0], qm, C)
        assert np.allclose(u, u0 + qm * e / C, rtol=0, atol=1e-15)


def test_boris_exb_drift_velocity(orc):
    """Crossed uniform fields with |E| < |B|: the guiding centre drifts with
    velocity c E x B / B^2 (cells per step in code units), for either charge."""
    ey, bz = 0.01, 0.05
    vd = C * ey / bz  # E x B = (Ey Bz, 0, 0)
    for qm in (1.0, -1.0):
        u = np.zeros(3)
        x = 0.0
        xs = []
        nsteps = 40000
        for _ in range(nsteps):
            u = orc.boris(u, [0, ey, 0], [0, 0, bz], qm, C)
            x += C * u[0] / math.sqrt(1.0 + u @ u)
            xs.append(x)
        xs = np.array(xs)
        # least-squares slope removes the bounded gyration
        t = np.arange(1, nsteps + 1)
        slope = np.polyfit(t, xs, 1)[0]
        assert abs(slope - vd) / vd < 2e-3


# ---------------------------------------------------------------- gather ----

def _grid(dim):
    return (16, 12, 10)[:dim] + (1,) * (3 - dim)


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_gather_reproduces_linear_fields(orc, dim):
    """Linear interpolation is exact for fields that are linear in position;
    each component is sampled at its own Yee point (Sect. 2.3.1)."""
    nx, ny, nz = _grid(dim)
    g = orc.Grid(dim, nx, ny, nz, C)
    rs = np.random.default_rng(5)
    a = rs.normal(size=6)
    b = rs.normal(size=(6, 3))
    F = g.zeros()
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    idx = (ii, jj, kk)
    for comp in range(6):
        st = (E_STAG + B_STAG)[comp]
        F[comp] = a[comp] + sum(b[comp, d] * (idx[d] + st[d]) for d in range(dim))
    ext = (nx, ny, nz)
    for _ in range(50):
        x = np.zeros(3)
        for d in range(dim):  # stay clear of the periodic seam
            x[d] = rs.uniform(1.0, ext[d] - 2.0)
        e, bb = orc.interp(g, F, x)
        got = np.concatenate([e, bb])
        expect = a + b[:, :dim] @ x[:dim]
        assert np.allclose(got, expect, rtol=0, atol=1e-12)


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_gather_impulse_is_tent_function(orc, dim):
    """A single nonzero lattice value is seen by a particle through the
    first-order (tent) shape centred on that component's Yee point, including
    across the periodic seam."""
    nx, ny, nz = _grid(dim)
    g = orc.Grid(dim, nx, ny, nz, C)
    ext = (nx, ny, nz)
    rs = np.random.default_rng(6)
    for comp in range(6):
        st = (E_STAG + B_STAG)[comp]
        F = g.zeros()
        p = (0, ny - 1, 3)[:dim] + (0,) * (3 - dim)  # i = 0 sits on the seam
        F[comp, p[2], p[1], p[0]] = 1.0
        for _ in range(40):
            x = np.zeros(3)
            for d in range(dim):
                x[d] = (p[d] + st[d] + rs.uniform(-1.2, 1.2)) % ext[d]
            e, b = orc.interp(g, F, x)
            got = np.concatenate([e, b])[comp]
            w = 1.0
            for d in range(dim):
                dist = (x[d] - (p[d] + st[d])) % ext[d]
                dist = min(dist, ext[d] - dist)
                w *= max(0.0, 1.0 - dist)
            assert abs(got - w) < 1e-12
            others = np.delete(np.concatenate([e, b]), comp)
            assert np.all(others == 0.0)


# ---------------------------------------------------------------- ZigZag ----

def _load_zigzag_cases():
    with open(os.path.join(GOLDEN, "zigzag_hand_sums.json")) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _load_zigzag_cases(), ids=lambda c: c["name"])
def test_zigzag_hand_sums(orc, case):
    """Hand-derived currents of one particle (Appendix D), every lattice value."""
    nx, ny, nz = case["n"]
    g = orc.Grid(case["dim"], nx, ny, nz, C)
    F = g.zeros()
    orc.zigzag(g, F, case["x1"], case["x2"], case["q"])
    expect = np.zeros((3,) + g.shape)
    for comp, i, j, k, v in case["J"]:
        expect[comp, k, j, i] += v
    assert np.allclose(F[6:9], expect, rtol=0, atol=1e-14)
    assert np.all(F[:6] == 0)


def _div_j(orc, g, F):
    G = g.zeros()
    G[0:3] = F[6:9]
    return orc.div_e(g, G)


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_zigzag_discrete_continuity(orc, dim):
    """rho(x2) - rho(x1) + div^- J = 0 on every node (Appendix B) for random
    moves of up to 0.45 cells per axis, with and without cell crossings and
    across the periodic seam."""
    nx, ny, nz = (9, 7, 6)[:dim] + (1,) * (3 - dim)
    g = orc.Grid(dim, nx, ny, nz, C)
    rs = np.random.default_rng(7)
    n = 400
    ext = np.array([nx, ny, nz], dtype=np.float64)
    x1 = np.zeros((3, n))
    x1[:dim] = rs.uniform(0, 1, size=(dim, n)) * ext[:dim, None]
    dx = rs.uniform(-0.45, 0.45, size=(3, n))
    q = rs.choice([-1.3, 0.7], size=n)
    F = g.zeros()
    for p in range(n):
        orc.zigzag(g, F, x1[:, p], x1[:, p] + dx[:, p], q[p])
    x2 = x1 + dx
    x2[:dim] %= ext[:dim, None]
    rho1 = sum(orc.charge_density(g, [orc.Species(q[p], 1, x1[:, p:p + 1], np.zeros((3, 1)))])
               for p in range(n))
    rho2 = sum(orc.charge_density(g, [orc.Species(q[p], 1, x2[:, p:p + 1], np.zeros((3, 1)))])
               for p in range(n))
    res = rho2 - rho1 + _div_j(orc, g, F)
    assert np.abs(res).max() < 1e-12


def test_zigzag_total_current_is_charge_times_displacement(orc):
    """Summed over the lattice, each component of the ZigZag current equals
    q times the displacement (both segments together cover x1 -> x2)."""
    g = orc.Grid(3, 6, 5, 4, C)
    rs = np.random.default_rng(8)
    for _ in range(30):
        x1 = rs.uniform(0, 1, 3) * np.array([6, 5, 4])
        d = rs.uniform(-0.45, 0.45, 3)
        F = g.zeros()
        orc.zigzag(g, F, x1, x1 + d, 0.8)
        assert np.allclose(F[6:9].reshape(3, -1).sum(axis=1), 0.8 * d, rtol=0, atol=1e-14)


@pytest.mark.parametrize("case", _load_zigzag_cases(), ids=lambda c: c["name"])
def test_zigzag_term_magnitudes_of_one_move_are_its_hand_sums(orc, case):
    """deposit_abs of a single move equals |J| of the hand sums: every term of
    one move on one component has the sign of its displacement."""
    nx, ny, nz = case["n"]
    g = orc.Grid(case["dim"], nx, ny, nz, C)
    A = g.zeros()
    x1 = np.asarray(case["x1"], dtype=np.float64).reshape(3, 1)
    dx = np.asarray(case["x2"], dtype=np.float64).reshape(3, 1) - x1
    orc.deposit_abs(g, A, x1, dx, case["q"])
    expect = np.zeros((3,) + g.shape)
    for comp, i, j, k, v in case["J"]:
        expect[comp, k, j, i] += v
    assert np.allclose(A[6:9], np.abs(expect), rtol=0, atol=1e-14)
    assert np.all(A[:6] == 0)


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_zigzag_term_magnitudes_bound_the_current(orc, dim):
    """Many moves of both charge signs: deposit_abs >= |deposit| on every word
    (the triangle inequality), and per component its lattice sum is
    sum_p |q_p| |dx_p| (each move's weights sum to one per segment; the 3D
    +-D_b D_c / 12 corrections cancel over a segment's four words)."""
    nx, ny, nz = (9, 7, 6)[:dim] + (1,) * (3 - dim)
    g = orc.Grid(dim, nx, ny, nz, C)
    rs = np.random.default_rng(70 + dim)
    n = 300
    ext = np.array([nx, ny, nz], dtype=np.float64)
    x1 = np.zeros((3, n))
    x1[:dim] = rs.uniform(0, 1, size=(dim, n)) * ext[:dim, None]
    dx = rs.uniform(-0.45, 0.45, size=(3, n))
    q = rs.choice([-1.3, 0.7], size=n)
    J, A = g.zeros(), g.zeros()
    for p in range(n):
        orc.deposit(g, J, x1[:, p:p + 1].copy(), dx[:, p:p + 1].copy(), q[p])
        orc.deposit_abs(g, A, x1[:, p:p + 1].copy(), dx[:, p:p + 1].copy(), q[p])
    assert np.all(A[6:9] >= np.abs(J[6:9]) - 1e-14)
    assert np.abs(J[6:9]).sum() < A[6:9].sum()  # charges of both signs cancel somewhere
    tot = (np.abs(q)[None, :] * np.abs(dx)).sum(axis=1)
    assert np.allclose(A[6:9].reshape(3, -1).sum(axis=1), tot, rtol=1e-12, atol=0)


# ---------------------------------------------------------------- FDTD2 -----

def _k_operator(kvec, order=2):
    """Symbol of the staggered difference: 2 sin(k/2) (second order) or
    2 [(9/8) sin(k/2) - (1/24) sin(3k/2)] (fourth order)."""
    k = np.asarray(kvec, dtype=np.float64)
    if order == 2:
        return 2.0 * np.sin(k / 2.0)
    return 2.0 * (9.0 / 8.0 * np.sin(k / 2.0) - 1.0 / 24.0 * np.sin(1.5 * k))


def _plane_wave(g, kvec, e_hat, t_e, order=2):
    """Discrete plane wave of the Yee scheme at E time t_e (B at t_e - 1/2).
    With K the symbol of the staggered difference and Omega = 2 sin(w/2), the
    update equations of Eqs. (fdE), (fdB) give Omega^2 = c^2 |K|^2 and
    b = c (K x e) / Omega for e orthogonal to K (the textbook Yee dispersion
    relation for K_d = 2 sin(k_d/2))."""
    K = _k_operator(kvec, order)
    om = 2.0 * math.asin(C * np.linalg.norm(K) / 2.0)
    b_hat = C * np.cross(K, e_hat) / (2.0 * math.sin(om / 2.0))
    F = g.zeros()
    kk, jj, ii = np.meshgrid(np.arange(g.nz), np.arange(g.ny), np.arange(g.nx), indexing="ij")
    idx = (ii, jj, kk)
    for a in range(3):
        pe = sum(kvec[d] * (idx[d] + E_STAG[a][d]) for d in range(3))
        pb = sum(kvec[d] * (idx[d] + B_STAG[a][d]) for d in range(3))
        F[a] = e_hat[a] * np.cos(pe - om * t_e)
        F[3 + a] = b_hat[a] * np.cos(pb - om * (t_e - 0.5))
    return F, om


@pytest.mark.parametrize("dim,modes", [(1, (3, 0, 0)), (2, (2, 5, 0)), (3, (1, 2, 3))])
def test_fdtd2_vacuum_plane_wave_dispersion(orc, dim, modes):
    """Vacuum: B half step, B half step, E step (J = 0) advance the Yee plane
    wave exactly along its numerical dispersion relation
    sin^2(w/2) = c^2 sum_d sin^2(k_d/2)."""
    nx, ny, nz = (32, 24, 16)[:dim] + (1,) * (3 - dim)
    g = orc.Grid(dim, nx, ny, nz, C)
    kvec = np.array([2 * math.pi * modes[0] / nx, 2 * math.pi * modes[1] / ny,
                     2 * math.pi * modes[2] / nz])
    K = 2.0 * np.sin(kvec / 2.0)
    # a unit polarisation orthogonal to K (discretely transverse wave)
    trial = np.array([0.3, -0.5, 0.8])
    e_hat = trial - K * (trial @ K) / (K @ K)
    e_hat /= np.linalg.norm(e_hat)
    F, _ = _plane_wave(g, kvec, e_hat, 0.0)
    nsteps = 40
    for _ in range(nsteps):
        orc.push_half_b(g, F)
        orc.push_half_b(g, F)
        orc.push_e(g, F)
    expect, _ = _plane_wave(g, kvec, e_hat, float(nsteps))
    assert np.abs(F[:6] - expect[:6]).max() < 1e-11


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_fdtd2_preserves_div_b_and_vacuum_div_e(orc, dim):
    """div^+ B and (with J = 0) div^- E are constants of the Yee update
    (Appendix B)."""
    nx, ny, nz = (10, 9, 8)[:dim] + (1,) * (3 - dim)
    g = orc.Grid(dim, nx, ny, nz, C)
    F = g.zeros()
    F[:6] = np.random.default_rng(9).normal(size=(6,) + g.shape)
    db0, de0 = orc.div_b(g, F), orc.div_e(g, F)
    for _ in range(25):
        orc.push_half_b(g, F)
        orc.push_half_b(g, F)
        orc.push_e(g, F)
    assert np.abs(orc.div_b(g, F) - db0).max() < 1e-11
    assert np.abs(orc.div_e(g, F) - de0).max() < 1e-11


# ------------------------------------------------------------- Binomial2 ----

@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("passes", [1, 2, 4])
def test_binomial_impulse_response(orc, dim, passes):
    """p passes of (1/4, 1/2, 1/4) per axis turn an impulse into the product of
    binomial coefficients C(2p, m) / 4^p (exact in binary floating point)."""
    nx, ny, nz = (16, 14, 12)[:dim] + (1,) * (3 - dim)
    g = orc.Grid(dim, nx, ny, nz, C)
    F = g.zeros()
    src = (1, 6, 5)  # i = 1 puts the response across the periodic seam
    for a in range(3):
        F[6 + a, src[2] if dim > 2 else 0, src[1] if dim > 1 else 0, src[0]] = 2.0 - a
    orc.filter_binomial(g, F, passes)
    w1 = np.array([math.comb(2 * passes, m) for m in range(2 * passes + 1)]) / 4.0**passes
    for a in range(3):
        expect = np.zeros(g.shape)
        for off in np.ndindex(*(len(w1),) * dim):
            wt = 2.0 - a
            pos = [0, 0, 0]
            for d in range(dim):
                wt *= w1[off[d]]
                pos[d] = (src[d] + off[d] - passes) % (nx, ny, nz)[d]
            expect[pos[2], pos[1], pos[0]] += wt
        assert np.array_equal(F[6 + a], expect)
    assert np.all(F[:6] == 0)


def test_binomial_fourier_response_and_mean(orc):
    """A lattice Fourier mode m along an axis of N cells is multiplied by
    cos^2(pi m / N) per pass; the k = 0 mode (the total current) is kept."""
    g = orc.Grid(2, 24, 20, 1, C)
    jj, ii = np.meshgrid(np.arange(20), np.arange(24), indexing="ij")
    mx, my = 5, 3
    F = g.zeros()
    F[6, 0] = np.cos(2 * math.pi * mx * ii / 24 + 0.3) * np.cos(2 * math.pi * my * jj / 20 - 1.1)
    F[7, 0] = 1.5 + np.cos(2 * math.pi * mx * ii / 24)
    F[8, 0] = np.random.default_rng(10).normal(size=(20, 24))
    s8 = F[8].sum()
    orc.filter_binomial(g, F, 3)
    fx = math.cos(math.pi * mx / 24) ** 2
    fy = math.cos(math.pi * my / 20) ** 2
    expect6 = (fx * fy) ** 3 * np.cos(2 * math.pi * mx * ii / 24 + 0.3) * \
        np.cos(2 * math.pi * my * jj / 20 - 1.1)
    assert np.abs(F[6, 0] - expect6).max() < 1e-13
    assert np.abs(F[7, 0] - (1.5 + fx**3 * np.cos(2 * math.pi * mx * ii / 24))).max() < 1e-13
    assert abs(F[8].sum() - s8) < 1e-11


# --------------------------------------------------------- Higuera-Cary ----

@pytest.mark.parametrize("beta_d", [0.3, 0.9, 0.99])
def test_higuera_cary_keeps_relativistic_exb_drift_exactly(orc, beta_d):
    """A particle moving with the E x B drift velocity feels no force; the
    Higuera-Cary rotation factor makes the discrete update keep it exactly,
    at any drift speed (Boris does not once the drift is relativistic)."""
    bz = 0.3
    ey = beta_d * bz  # E + (u/gamma) x B = 0 for u/gamma = beta_d x-hat
    gam = 1.0 / math.sqrt(1.0 - beta_d**2)
    u0 = np.array([gam * beta_d, 0.0, 0.0])
    for qm in (1.0, -1.0):
        u = u0.copy()
        for _ in range(200):
            u = orc.higuera_cary(u, [0, ey, 0], [0, 0, bz], qm, C)
        assert np.abs(u - u0).max() < 1e-11
    ub = orc.boris(u0, [0, ey, 0], [0, 0, bz], 1.0, C)
    if beta_d >= 0.9:
        assert np.abs(ub - u0).max() > 1e-4  # the closed form separates the two pushers


def test_higuera_cary_rotation_and_pure_kick(orc):
    """E = 0: the update is a rotation (|u| kept); B = 0: the two half kicks
    add to u + s E / c exactly, as for Boris."""
    u0 = np.array([1.7, -0.6, 0.4])
    u = u0.copy()
    for _ in range(300):
        u = orc.higuera_cary(u, [0, 0, 0], [0.1, -0.2, 0.9], -1.0, C)
    assert abs(np.linalg.norm(u) - np.linalg.norm(u0)) < 1e-12
    e = np.array([0.01, -0.02, 0.03])
    assert np.allclose(orc.higuera_cary(u0, e, [0, 0, 0], 1.0, C), u0 + e / C, rtol=0, atol=1e-15)


@pytest.mark.parametrize("dim,modes", [(1, (3, 0, 0)), (2, (2, 5, 0)), (3, (1, 2, 3))])
def test_fdtd4_vacuum_plane_wave_dispersion(orc, dim, modes):
    """FDTD4 (Table 2): the fourth-order staggered differences advance a
    plane wave exactly along sin^2(w/2) = (c^2/4) sum_d K4_d^2,
    K4 = 2 [(9/8) sin(k/2) - (1/24) sin(3k/2)]."""
    nx, ny, nz = (32, 24, 16)[:dim] + (1,) * (3 - dim)
    g = orc.Grid(dim, nx, ny, nz, C)
    kvec = np.array([2 * math.pi * modes[0] / nx, 2 * math.pi * modes[1] / ny,
                     2 * math.pi * modes[2] / nz])
    K = _k_operator(kvec, 4)
    trial = np.array([0.3, -0.5, 0.8])
    e_hat = trial - K * (trial @ K) / (K @ K)
    e_hat /= np.linalg.norm(e_hat)
    F, _ = _plane_wave(g, kvec, e_hat, 0.0, order=4)
    orc.set_field_order(4)
    try:
        for _ in range(40):
            orc.push_half_b(g, F)
            orc.push_half_b(g, F)
            orc.push_e(g, F)
    finally:
        orc.set_field_order(2)
    expect, _ = _plane_wave(g, kvec, e_hat, 40.0, order=4)
    assert np.abs(F[:6] - expect[:6]).max() < 1e-11
    # the second-order wave differs: the test separates the two solvers
    expect2, _ = _plane_wave(g, kvec, e_hat, 40.0, order=2)
    assert np.abs(F[:6] - expect2[:6]).max() > 1e-6
