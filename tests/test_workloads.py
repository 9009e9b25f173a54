"""The seeded input recipes (workloads/) against the definitions of the
paper's set-ups.  Both the oracle and the CUDA path start from these inputs,
so a mistake here would pass every parity test: each recipe is checked
against an independent statement of what it must produce (a quadrature, a
physical definition, a discrete identity, a sample statistic)."""
import math

import numpy as np
import pytest
from scipy import integrate

import workloads
from workloads.plasma import ONE_MINUS


@pytest.mark.parametrize("theta", [0.01, 0.1, 0.3, 1.0])
def test_mean_lorentz_factor_matches_quadrature_of_the_maxwell_juettner_law(theta):
    """<gamma> of f(p) ~ p^2 exp(-(gamma - 1)/theta), integrated numerically."""
    def f(p, w):
        g = math.sqrt(1.0 + p * p)
        return w(g) * p * p * math.exp(-(g - 1.0) / theta)

    top = math.sqrt((1.0 + 80.0 * theta) ** 2 - 1.0)
    num = integrate.quad(f, 0.0, top, args=(lambda g: g,), limit=400, epsabs=0, epsrel=1e-12)[0]
    den = integrate.quad(f, 0.0, top, args=(lambda g: 1.0,), limit=400, epsabs=0, epsrel=1e-12)[0]
    assert workloads.mj_mean_gamma(theta) == pytest.approx(num / den, rel=1e-9)


def test_maxwell_juettner_sample_mean_and_isotropy():
    gen = workloads.plasma.rng(11)
    theta, n = 0.3, 400_000
    u = workloads.sample_mj_momenta(gen, n, theta)
    g = np.sqrt(1.0 + (u * u).sum(0))
    # sample mean of gamma within 5 standard errors of the distribution's mean
    assert abs(g.mean() - workloads.mj_mean_gamma(theta)) < 5.0 * g.std() / math.sqrt(n)
    # isotropic: no mean momentum, equal second moments per axis
    for a in range(3):
        assert abs(u[a].mean()) < 5.0 * u[a].std() / math.sqrt(n)
    m2 = (u * u).mean(1)
    assert np.abs(m2 / m2.mean() - 1.0).max() < 0.01


def test_cold_boost_gives_the_drift_four_velocity():
    """A cold gas boosted to beta along an axis has u = Gamma beta there."""
    gen = workloads.plasma.rng(12)
    u = workloads.sample_mj_momenta(gen, 10_000, 1e-8)
    beta = 0.6
    ub = workloads.boost_flip(gen, u, 1, beta)
    big = 1.0 / math.sqrt(1.0 - beta * beta)
    assert np.abs(ub[1] - big * beta).max() < 1e-3
    assert np.abs(ub[0]).max() < 1e-3 and np.abs(ub[2]).max() < 1e-3


def test_pairs_share_positions_and_cancel_charge():
    pl = workloads.uniform_plasma(2, 12, 9, 1, 0.45, 6, 0.01, 0.2, seed=3)
    e, p = pl.species
    assert e.q == -p.q and e.m == p.m == abs(e.q)
    assert np.array_equal(e.cell, p.cell) and np.array_equal(e.off, p.off)
    assert not np.array_equal(e.u, p.u)  # velocities drawn independently
    # every cell holds ppc particles of each species, offsets in [0, 1)
    assert np.array_equal(np.bincount(e.cell, minlength=12 * 9), np.full(12 * 9, 6))
    assert e.off.dtype == np.float32 and (e.off >= 0).all() and (e.off <= ONE_MINUS).all()


def test_charge_gives_the_skin_depth_through_the_plasma_frequency():
    """Code units (4 pi absorbed, unit cell volume): w_p^2 = sum_s n_s q_s^2 /
    (m_s <gamma>) must equal (c / R_p)^2 for the Weibel box (<gamma> =
    gamma_b)."""
    pl = workloads.weibel_1d(nx=16, ppc=8, gamma_b=3.0, theta=0.01, r_p=10.0)
    n_s = 8.0  # particles per cell per species
    wp2 = sum(n_s * s.q * s.q / (s.m * 3.0) for s in pl.species)
    assert wp2 == pytest.approx((0.45 / 10.0) ** 2, rel=1e-12)


def test_weibel_beams_carry_half_of_each_species_each_way():
    pl = workloads.weibel_1d(nx=32, ppc=8, gamma_b=3.0, theta=1e-10)  # spread ~3e-5
    gb = 3.0 * math.sqrt(1.0 - 1.0 / 9.0)  # gamma_b beta_b
    for s in pl.species:
        uy = s.u[1].astype(np.float64)
        up, down = uy > 0, uy < 0
        assert up.sum() == down.sum() == s.n // 2
        assert np.abs(np.abs(uy) - gb).max() < 1e-3 * gb
        assert np.abs(s.u[0]).max() < 1e-3 and np.abs(s.u[2]).max() < 1e-3


def test_turbulence_guide_field_gives_sigma_and_the_forcing_is_solenoidal():
    pl = workloads.turbulence_2d(n=64, ppc=4, r_p=4.0, theta=0.3, sigma=10.0, modes=4, seed=5)
    F = pl.fields.astype(np.float64)
    b0 = F[5, 0, 0, 0]
    assert np.all(F[5] == F[5, 0, 0, 0])  # uniform guide field along z
    # magnetisation: sigma = B0^2 / (sum_s n_s m_s c^2 <gamma>), both species
    g = workloads.mj_mean_gamma(0.3)
    enthalpy = sum(4.0 * s.m * 0.45 ** 2 * g for s in pl.species)
    assert b0 * b0 / enthalpy == pytest.approx(10.0, rel=1e-6)
    # Bx at (i, j+1/2), By at (i+1/2, j): div+ B at the cell centres vanishes
    bx, by = F[3, 0], F[4, 0]
    div = (np.roll(bx, -1, axis=1) - bx) + (np.roll(by, -1, axis=0) - by)
    assert np.abs(div).max() < 1e-6 * max(np.abs(bx).max(), np.abs(by).max())
    # the in-plane perturbation has rms dB / B0 near the requested 1
    rms = math.sqrt((bx * bx + by * by).mean()) / b0
    assert 0.8 < rms < 1.2
    assert np.abs(F[0:3]).max() == 0.0 and np.abs(F[6:9]).max() == 0.0


def test_adjoint_modes_are_solenoidal_and_scaled():
    pl, mf, amps = workloads.adjoint_box(n=32, ppc=2, theta=0.1, sigma=1.0, modes=4, seed=9)
    assert mf.shape[0] == 16 and amps.shape == (16,)
    for m in mf.astype(np.float64):
        bx, by = m[0, 0], m[1, 0]
        div = (np.roll(bx, -1, axis=1) - bx) + (np.roll(by, -1, axis=0) - by)
        assert np.abs(div).max() < 1e-5 * max(np.abs(bx).max(), np.abs(by).max(), 1e-30)
        assert np.abs(m[2]).max() == 0.0  # in-plane perturbations only
    # the summed perturbation has rms |dB| = 0.1 B0 (B0 the guide field)
    b0 = float(pl.fields[5, 0, 0, 0])
    db = np.tensordot(amps.astype(np.float64), mf.astype(np.float64), axes=1)
    assert math.sqrt((db ** 2).sum(0).mean()) == pytest.approx(0.1 * b0, rel=1e-5)


def test_ensemble_recipe_stays_in_its_ranges():
    boxes = workloads.weibel_ensemble(count=256)
    assert len(boxes) == 256
    dims = [b[0] for b in boxes]
    assert set(dims) == {1, 2}
    for dim, n, ppc, gamma_b, theta, seed in boxes:
        assert (128 <= n <= 4096) if dim == 1 else (32 <= n <= 256)
        assert 16 <= ppc <= 128 and ppc % 2 == 0
        assert 1.5 <= gamma_b <= 10.0 and 0.001 <= theta <= 0.1


def test_recipes_are_seeded():
    a = workloads.uniform_plasma(3, 5, 4, 3, 0.45, 2, 0.01, 0.1, seed=21)
    b = workloads.uniform_plasma(3, 5, 4, 3, 0.45, 2, 0.01, 0.1, seed=21)
    c = workloads.uniform_plasma(3, 5, 4, 3, 0.45, 2, 0.01, 0.1, seed=22)
    for x, y, z in zip(a.species, b.species, c.species):
        assert np.array_equal(x.off, y.off) and np.array_equal(x.u, y.u)
        assert not np.array_equal(x.u, z.u)
