"""Whole-step pins of the FP64 oracle: discrete Gauss law (Appendix B), energy
bookkeeping, the Weibel growth rate of Sect. 4.1 and the sorted-layout
definition.  No CUDA code is involved."""
import math

import numpy as np
import pytest

import workloads


def _small_turbulence(n=32, ppc=4, seed=11):
    return workloads.turbulence_2d(n=n, ppc=ppc, r_p=4.0, theta=0.3, sigma=1.0,
                                   db_over_b0=1.0, modes=4, seed=seed)


@pytest.mark.parametrize("passes", [0, 2])
def test_gauss_law_at_round_off_2d(orc, passes):
    """With co-located pairs rho = 0 and div E = 0 at t = 0; the Yee update plus
    charge-conserving deposit keep div E - F^p(rho) = 0 (the Binomial2 filter F
    commutes with the divergence) to round-off."""
    pl = _small_turbulence()
    g, F, sp = orc.from_plasma(pl)
    assert np.abs(orc.gauss_residual(g, F, sp, passes)).max() < 1e-15
    scale = 0.0
    for _ in range(30):
        orc.step(g, F, sp, passes=passes)
        scale = max(scale, np.abs(orc.div_e(g, F)).max())
    res = np.abs(orc.gauss_residual(g, F, sp, passes)).max()
    assert scale > 1e-6  # the test is not vacuous: charge separation happened
    assert res < 1e-13 * max(1.0, scale / 1e-3)


def test_gauss_law_at_round_off_3d(orc):
    pl = workloads.uniform_plasma(3, 8, 6, 5, 0.45, 2, 0.01, 0.2, seed=12)
    g, F, sp = orc.from_plasma(pl)
    for _ in range(15):
        orc.step(g, F, sp, passes=1)
    assert np.abs(orc.div_e(g, F)).max() > 1e-6
    assert np.abs(orc.gauss_residual(g, F, sp, 1)).max() < 1e-14


def test_div_b_kept_by_full_step(orc):
    """div^+ B of the turbulence forcing (a discrete curl) is 0 and stays 0."""
    pl = _small_turbulence()
    g, F, sp = orc.from_plasma(pl)
    b0 = np.abs(orc.div_b(g, F)).max()
    assert b0 < 1e-6  # FP32-rounded initial field
    for _ in range(10):
        orc.step(g, F, sp)
    assert np.abs(orc.div_b(g, F)).max() < b0 + 1e-12


def test_energy_exchange_matches_field_work(orc):
    """Over one step the kinetic energy gained equals, to second order in the
    field, the work -sum E.J of the current on the field: the total
    0.5 sum (E^2 + B^2) + sum m c^2 (gamma - 1) drifts by far less than the
    energy that is exchanged."""
    pl = workloads.weibel_1d(nx=64, ppc=32, seed=13)
    g, F, sp = orc.from_plasma(pl)
    e0 = orc.energies(g, F, sp)
    for _ in range(120):
        orc.step(g, F, sp)
    e1 = orc.energies(g, F, sp)
    exchanged = abs(e1[1] - e0[1]) + abs(e1[0] - e0[0])
    assert exchanged > 0
    assert abs(sum(e1) - sum(e0)) < 0.05 * exchanged


def test_weibel_linear_growth_rate(orc):
    """Sect. 4.1: the filamentation growth rate of symmetric beams is
    delta / w_p = beta_b sqrt(2 / gamma_b) (Bret 2010), w_p = c / R_p per step
    in code units, so the magnetic energy grows as exp(2 delta t).  The run is
    the 1D3V box of 512 cells, 64 particles per cell per species, gamma_b = 3,
    theta = 0.01.  Warm beams and the finite wave numbers of the box lower the
    cold-beam maximum, so the fitted rate must lie within 0.85-1.02 of 2 delta."""
    pl = workloads.weibel_1d()
    g, F, sp = orc.from_plasma(pl)
    m = pl.meta
    delta = m["beta_b"] * math.sqrt(2.0 / m["gamma_b"]) * g.c / m["r_p"]
    eb = []
    for _ in range(230):
        orc.step(g, F, sp)
        eb.append(orc.field_energy(g, F)[1])
    eb = np.array(eb)
    t = np.arange(1, len(eb) + 1)
    sat = eb.max()
    end = np.argmax(eb > 0.5 * sat)
    win = (eb > 3e-4 * sat) & (eb < 3e-2 * sat) & (t < t[end])
    assert win.sum() > 30
    rate = np.polyfit(t[win], np.log(eb[win]), 1)[0]
    assert 0.85 * 2 * delta < rate < 1.02 * 2 * delta, (rate, 2 * delta)


def test_tile_sort_reference_is_stable_counting_sort(orc):
    """Brute force on a small input: the permutation is the stable sort by tile
    key and the offsets count each tile's particles."""
    rs = np.random.default_rng(14)
    nx, ny, nz, tile = 10, 7, 3, (4, 3, 2)
    cell = rs.integers(0, nx * ny * nz, size=300).astype(np.int32)
    perm, start = orc.tile_sort_reference(cell, nx, ny, nz, tile)

    def key(c):
        i, j, k = c % nx, (c // nx) % ny, c // (nx * ny)
        return (i // 4) + 3 * ((j // 3) + 3 * (k // 2))

    brute = sorted(range(len(cell)), key=lambda p: (key(int(cell[p])), p))
    assert list(perm) == brute
    ntiles = 3 * 3 * 2
    assert start[0] == 0 and start[-1] == len(cell) and len(start) == ntiles + 1
    for t in range(ntiles):
        assert start[t + 1] - start[t] == sum(1 for c in cell if key(int(c)) == t)
