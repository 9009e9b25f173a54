"""Pins of the oracle's discrete adjoint (reverse mode of the time step):
transposes of the field updates by the dot-product identity, and the full
step's gradient against central finite differences of the oracle's own
forward step (double precision), in 1D, 2D and 3D, with and without the
filter, over one and several steps.  No CUDA code is involved."""
import numpy as np
import pytest

C = 0.45


def _fields(orc, g, rs, amp_e=0.02, amp_b=0.05):
    F = g.zeros()
    F[0:3] = amp_e * rs.normal(size=(3,) + g.shape)
    F[3:6] = amp_b * rs.normal(size=(3,) + g.shape)
    return F


def _particles(orc, g, rs, n, q, m):
    x = np.zeros((3, n))
    for d in range(g.dim):
        x[d] = rs.uniform(2.0, g.extents()[d] - 2.0, n)  # no wrap within a few steps
    u = rs.normal(0.0, 1.2, (3, n))
    return orc.Species(q, m, x, u)


def _state(orc, dim, seed):
    g = orc.Grid(dim, *((10, 7, 6)[:dim] + (1,) * (3 - dim)), C)
    rs = np.random.default_rng(seed)
    F = _fields(orc, g, rs)
    sp = [_particles(orc, g, rs, 30, -0.05, 0.05), _particles(orc, g, rs, 25, 0.08, 0.08)]
    return g, F, sp


def _copy(orc, F, sp):
    return F.copy(), [orc.Species(s.q, s.m, s.x.copy(), s.u.copy()) for s in sp]


def _loss(orc, g, F, sp, lam, nsteps, passes):
    F, sp = _copy(orc, F, sp)
    orc.step(g, F, sp, passes=passes, nsteps=nsteps)
    lF, lx, lu = lam
    v = float((lF[0:6] * F[0:6]).sum())
    for s, a, b in zip(sp, lx, lu):
        v += float((a[: g.dim] * s.x[: g.dim]).sum() + (b * s.u).sum())
    return v


def test_field_update_adjoints_are_transposes(orc):
    """<M f, a> = <f, M^T a> for the B half step and the E update with -J."""
    g = orc.Grid(3, 6, 5, 4, C)
    rs = np.random.default_rng(3)
    f, a = rs.normal(size=(9,) + g.shape), rs.normal(size=(9,) + g.shape)
    a[6:9] = 0.0
    mf = f.copy()
    orc.push_half_b(g, mf)
    ma = a.copy()
    orc.lib().orc_adj_push_half_b(g.c_struct(), orc._p(ma))
    assert (mf[0:6] * a[0:6]).sum() == pytest.approx((f[0:6] * ma[0:6]).sum(), rel=1e-12)
    mf = f.copy()
    orc.push_e(g, mf)
    orc.add_cur(g, mf)
    ma = a.copy()
    orc.lib().orc_adj_push_e(g.c_struct(), orc._p(ma))
    assert (mf[0:6] * a[0:6]).sum() == pytest.approx((f * ma).sum(), rel=1e-12)


@pytest.mark.parametrize("dim,passes,nsteps", [(1, 0, 1), (2, 0, 1), (2, 2, 1), (3, 1, 1),
                                               (1, 0, 3), (2, 1, 3), (3, 0, 2)])
def test_step_gradient_matches_central_differences(orc, dim, passes, nsteps):
    """L = <lambda, state after nsteps>; the adjoint's <grad, delta> equals
    (L(s + h delta) - L(s - h delta)) / 2h along random directions delta of
    E, B, every position and every four-velocity."""
    g, F, sp = _state(orc, dim, 20 + 10 * dim + nsteps)
    rs = np.random.default_rng(7 + dim)
    lam = (rs.normal(size=(9,) + g.shape), [rs.normal(size=(3, s.n)) for s in sp],
           [rs.normal(size=(3, s.n)) for s in sp])
    for s in lam[1]:
        s[dim:] = 0.0

    def loss_grad(Ff, spf):
        A = lam[0].copy()
        A[6:9] = 0.0
        return A, [a.copy() for a in lam[1]], [b.copy() for b in lam[2]]

    F0, sp0 = _copy(orc, F, sp)
    A, xbar, ubar = orc.gradient(g, F, sp, nsteps, loss_grad, passes=passes)
    for trial in range(3):
        dF = rs.normal(size=F0.shape)
        dF[6:9] = 0.0
        dx = [rs.normal(size=(3, s.n)) for s in sp0]
        for d in dx:
            d[dim:] = 0.0
        du = [rs.normal(size=(3, s.n)) for s in sp0]
        pred = float((A[0:6] * dF[0:6]).sum())
        pred += sum(float((a * b).sum()) for a, b in zip(xbar, dx))
        pred += sum(float((a * b).sum()) for a, b in zip(ubar, du))
        h = 1e-7

        def shifted(sign):
            Fs, sps = _copy(orc, F0, sp0)
            Fs += sign * h * dF
            for s, a, b in zip(sps, dx, du):
                s.x += sign * h * a
                s.u += sign * h * b
            return _loss(orc, g, Fs, sps, lam, nsteps, passes)

        fd = (shifted(1.0) - shifted(-1.0)) / (2 * h)
        assert pred == pytest.approx(fd, rel=2e-6, abs=1e-8), (trial, pred, fd)


def test_magnetic_energy_gradient_of_a_weibel_run(orc):
    """Gradient of 0.5 sum B^2 after 6 steps of a small 1D Weibel plasma with
    respect to single four-velocity components and single field values,
    against central differences."""
    import workloads

    pl = workloads.weibel_1d(nx=24, ppc=4, gamma_b=3.0, theta=0.05, r_p=2.0, seed=5)
    g, F, sp = orc.from_plasma(pl)
    F[3:6] += 1e-3 * np.random.default_rng(9).normal(size=(3,) + g.shape)  # seed the instability

    def loss_grad(Ff, spf):
        A = g.zeros()
        A[3:6] = Ff[3:6]
        return A, [np.zeros((3, s.n)) for s in spf], [np.zeros((3, s.n)) for s in spf]

    F0, sp0 = _copy(orc, F, sp)
    A, xbar, ubar = orc.gradient(g, F, sp, 6, loss_grad)

    def loss(Fs, sps):
        Fs, sps = _copy(orc, Fs, sps)
        orc.step(g, Fs, sps, nsteps=6)
        return 0.5 * float((Fs[3:6] ** 2).sum())

    h = 1e-6
    for s_idx, a, p in [(0, 1, 3), (1, 0, 17), (0, 2, 40)]:
        def at(sign):
            Fs, sps = _copy(orc, F0, sp0)
            sps[s_idx].u[a, p] += sign * h
            return loss(Fs, sps)
        fd = (at(1) - at(-1)) / (2 * h)
        assert ubar[s_idx][a, p] == pytest.approx(fd, rel=1e-5, abs=1e-12)
    for comp, i in [(4, 5), (1, 11)]:
        def atf(sign):
            Fs, sps = _copy(orc, F0, sp0)
            Fs[comp, 0, 0, i] += sign * h
            return loss(Fs, sps)
        fd = (atf(1) - atf(-1)) / (2 * h)
        assert A[comp, 0, 0, i] == pytest.approx(fd, rel=1e-5, abs=1e-12)


def test_adjoint_box_modes_are_solenoidal_and_scaled():
    """The perturbation modes of the differentiable set-up are lattice curls
    (div+ B = 0 at the cell centres) and the seeded amplitudes give the
    requested rms dB / B0."""
    import workloads

    pl, mf, amps = workloads.adjoint_box(n=32, ppc=2, modes=4, db_over_b0=0.1, seed=3)
    bx, by = mf[:, 0, 0].astype(np.float64), mf[:, 1, 0].astype(np.float64)
    div = (np.roll(bx, -1, axis=2) - bx) + (np.roll(by, -1, axis=1) - by)
    assert np.abs(div).max() < 1e-6
    db = np.tensordot(amps.astype(np.float64), mf.astype(np.float64), axes=1)
    assert np.sqrt((db ** 2).sum(0).mean()) == pytest.approx(0.1 * pl.meta["b0"], rel=1e-5)
