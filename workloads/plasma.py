"""Seeded initial conditions for pair-plasma PIC runs.

Layout of what is produced (identical bytes go to the GPU path and the oracle):

* particles, per species, structure of arrays:
    ``cell``  int32[N]      linear cell index i + nx*(j + ny*k)
    ``off``   float32[D, N] in-cell offset of each gridded coordinate, in [0, 1)
    ``u``     float32[3, N] spatial four-velocity in units of c
* fields: float32[9, nz, ny, nx] planes Ex, Ey, Ez, Bx, By, Bz, Jx, Jy, Jz on
  the Yee lattice of Sect. 2.3.1 (plane index [i, j, k] of Ex is the point
  (i+1/2, j, k), of Bx the point (i, j+1/2, k+1/2), and so on).

Code units follow Appendix A: dx = dt = 1, the Courant number c is the only
constant of the field equations, |q| = m for every macro-particle of a pair
plasma and the charge is fixed by the skin depth R_p (in cells).

Random numbers come from numpy's Philox counter-based generator, whose stream
is the same on every platform.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy import special

ONE_MINUS = np.nextafter(np.float32(1.0), np.float32(0.0))  # largest float32 < 1


@dataclasses.dataclass
class Species:
    """One particle species: charge q (signed, code units), mass m (code units)."""

    q: float
    m: float
    cell: np.ndarray  # int32[N]
    off: np.ndarray  # float32[D, N]
    u: np.ndarray  # float32[3, N]

    @property
    def n(self) -> int:
        return int(self.cell.shape[0])


@dataclasses.dataclass
class Plasma:
    """A periodic box: grid, Courant number, species and the 9 field planes."""

    dim: int
    nx: int
    ny: int
    nz: int
    c: float
    species: list
    fields: np.ndarray  # float32[9, nz, ny, nx]
    meta: dict

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def nparticles(self) -> int:
        return sum(s.n for s in self.species)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


def mj_mean_gamma(theta: float) -> float:
    """Mean Lorentz factor of a Maxwell-Juettner gas, K1(1/t)/K2(1/t) + 3t."""
    z = 1.0 / theta
    if z > 500.0:  # asymptotic form, avoids underflow of kv
        return 1.0 + 1.5 * theta + 15.0 / 8.0 * theta**2
    return float(special.kve(1, z) / special.kve(2, z) + 3.0 * theta)


def charge_from_skin_depth(c: float, r_p: float, ppc: int, mean_gamma: float,
                           mass_ratio_sum: float = 2.0) -> float:
    """|q| fixed by the skin depth (Appendix A): w_p0 = c / R_p and
    |q| = w_p0^2 <gamma> / (N_ppc (1 + m-/m+))."""
    wp0 = c / r_p
    return wp0 * wp0 * mean_gamma / (ppc * mass_ratio_sum)


def sample_mj_momenta(gen: np.random.Generator, n: int, theta: float) -> np.ndarray:
    """Isotropic Maxwell-Juettner four-velocities u (units of c), float64[3, n].

    |u| is drawn by inverting the tabulated cumulative distribution of
    p^2 exp(-(sqrt(1+p^2)-1)/theta); the direction is uniform on the sphere.
    The table spans the distribution out to gamma-1 = 60 theta."""
    pmax = math.sqrt((1.0 + 60.0 * theta) ** 2 - 1.0)
    p = np.linspace(0.0, pmax, 1 << 17)
    logg = 2.0 * np.log(np.maximum(p, 1e-300)) - (np.sqrt(1.0 + p * p) - 1.0) / theta
    g = np.exp(logg - logg.max())
    g[0] = 0.0
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (g[1:] + g[:-1]) * np.diff(p))])
    cdf /= cdf[-1]
    mag = np.interp(gen.random(n), cdf, p)
    cos_t = 2.0 * gen.random(n) - 1.0
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    phi = 2.0 * math.pi * gen.random(n)
    return np.stack([mag * sin_t * np.cos(phi), mag * sin_t * np.sin(phi), mag * cos_t])


def boost_flip(gen: np.random.Generator, u: np.ndarray, axis: int, beta: np.ndarray) -> np.ndarray:
    """Boost rest-frame momenta u (float64[3, n]) to drift velocity beta along
    `axis` with the flipping method of Zenitani (2015): a particle whose
    velocity component satisfies -beta v > X (X uniform) has that component
    reversed first, which reweights the rest-frame sample by (1 + beta v) as the
    Lorentz transformation of the number density requires; then
    u' = Gamma (u + beta gamma)."""
    beta = np.broadcast_to(np.asarray(beta, dtype=np.float64), u.shape[1:])
    gam = np.sqrt(1.0 + (u * u).sum(axis=0))
    ua = u[axis].copy()
    flip = -beta * (ua / gam) > gen.random(ua.shape[0])
    ua[flip] = -ua[flip]
    big = 1.0 / np.sqrt(1.0 - beta * beta)
    out = u.copy()
    out[axis] = big * (ua + beta * gam)
    return out


_CHUNK = 1 << 22  # particles drawn per chunk; fixed so the streams never change


def uniform_plasma(dim: int, nx: int, ny: int, nz: int, c: float, ppc: int,
                   q_abs: float, theta: float, seed: int,
                   drift_axis: int = 0, drift_beta_per_slot=None,
                   meta: dict | None = None) -> Plasma:
    """Electron-positron plasma, `ppc` particles per cell per species.

    Offsets are uniform in each cell; particle k of the electrons and particle k
    of the positrons share their position (so the initial charge density is 0
    exactly), their four-velocities are drawn independently.  The slot of a
    particle inside its cell (0..ppc-1) selects its drift velocity from
    `drift_beta_per_slot` (None = at rest), applied along `drift_axis`."""
    if dim == 1:
        ny = nz = 1
    elif dim == 2:
        nz = 1
    ncells = nx * ny * nz
    n = ncells * ppc
    gen = rng(seed)
    cell = np.repeat(np.arange(ncells, dtype=np.int32), ppc)
    off = np.empty((dim, n), dtype=np.float32)
    us = [np.empty((3, n), dtype=np.float32) for _ in range(2)]
    slot_beta = None
    if drift_beta_per_slot is not None:
        slot_beta = np.asarray(drift_beta_per_slot, dtype=np.float64)
        assert slot_beta.shape == (ppc,)
    for lo in range(0, n, _CHUNK):
        hi = min(n, lo + _CHUNK)
        o = gen.random((dim, hi - lo)).astype(np.float32)
        off[:, lo:hi] = np.minimum(o, ONE_MINUS)
        for s in range(2):
            u = sample_mj_momenta(gen, hi - lo, theta)
            if slot_beta is not None:
                beta = slot_beta[np.arange(lo, hi) % ppc]
                u = boost_flip(gen, u, drift_axis, beta)
            us[s][:, lo:hi] = u.astype(np.float32)
    species = [
        Species(q=-q_abs, m=q_abs, cell=cell, off=off, u=us[0]),
        Species(q=+q_abs, m=q_abs, cell=cell.copy(), off=off.copy(), u=us[1]),
    ]
    fields = np.zeros((9, nz, ny, nx), dtype=np.float32)
    return Plasma(dim=dim, nx=nx, ny=ny, nz=nz, c=c, species=species,
                  fields=fields, meta=dict(meta or {}))


def weibel_1d(nx: int = 512, ppc: int = 64, gamma_b: float = 3.0, theta: float = 0.01,
              r_p: float = 10.0, c: float = 0.45, seed: int = 1234) -> Plasma:
    """Relativistic Weibel (filamentation) set-up of Sect. 4.1 in 1D3V: wave
    vector along x, two counter-streaming beams along +-y with Lorentz factor
    gamma_b, each carrying half of every species; zero initial fields.
    Charge from Appendix A with <gamma> = gamma_b."""
    q_abs = charge_from_skin_depth(c, r_p, ppc, gamma_b)
    beta_b = math.sqrt(1.0 - 1.0 / gamma_b**2)
    slots = np.where(np.arange(ppc) < ppc // 2, beta_b, -beta_b)
    return uniform_plasma(1, nx, 1, 1, c, ppc, q_abs, theta, seed,
                          drift_axis=1, drift_beta_per_slot=slots,
                          meta=dict(workload="weibel_1d3v", gamma_b=gamma_b, beta_b=beta_b,
                                    theta=theta, r_p=r_p, ppc=ppc, q_abs=q_abs,
                                    filter_passes=0))


def turbulence_2d(n: int = 1024, ppc: int = 16, r_p: float = 4.0, theta: float = 0.3,
                  sigma: float = 10.0, db_over_b0: float = 1.0, modes: int = 8,
                  c: float = 0.45, seed: int = 1235) -> Plasma:
    """Decaying turbulence set-up of Sect. 4.3 in 2D3V: pair plasma at rest
    with Maxwell-Juettner temperature theta, guide field B0 z-hat from the
    magnetization sigma (Appendix A, both species' enthalpy), and in-plane
    perturbations summed over modes m, n = 1..`modes` with random phases and
    amplitudes beta_mn = 2 dB / (N sqrt(m^2+n^2)).

    The perturbation is the curl of A_z = sum beta_mn (L/2pi)
    sin(k_m x + phi) sin(k_n y + psi), differenced on the lattice, which gives the
    printed dBx, dBy in the continuum limit and a discretely solenoidal B."""
    mean_g = mj_mean_gamma(theta)
    q_abs = charge_from_skin_depth(c, r_p, ppc, mean_g)
    b0 = math.sqrt(sigma * ppc * q_abs * c * c * mean_g * 2.0)
    pl = uniform_plasma(2, n, n, 1, c, ppc, q_abs, theta, seed,
                        meta=dict(workload="turbulence_2d3v", theta=theta, sigma=sigma,
                                  r_p=r_p, ppc=ppc, q_abs=q_abs, b0=b0, mean_gamma=mean_g,
                                  filter_passes=0))
    gen = rng(seed + 100000)
    phi = 2.0 * math.pi * gen.random((modes, modes))
    psi = 2.0 * math.pi * gen.random((modes, modes))
    L = float(n)
    x = np.arange(n, dtype=np.float64)
    az = np.zeros((n, n), dtype=np.float64)  # [j, i]
    db = db_over_b0 * b0
    for m in range(1, modes + 1):
        for nn in range(1, modes + 1):
            beta = 2.0 * db / (modes * math.sqrt(m * m + nn * nn))
            sx = np.sin(2.0 * math.pi * m * x / L + phi[m - 1, nn - 1])
            sy = np.sin(2.0 * math.pi * nn * x / L + psi[m - 1, nn - 1])
            az += beta * (L / (2.0 * math.pi)) * np.outer(sy, sx)
    bx = np.roll(az, -1, axis=0) - az  # at (i, j+1/2)
    by = -(np.roll(az, -1, axis=1) - az)  # at (i+1/2, j)
    pl.fields[3, 0] = bx.astype(np.float32)
    pl.fields[4, 0] = by.astype(np.float32)
    pl.fields[5, 0] = np.float32(b0)
    pl.meta["db_rms_over_b0"] = float(np.sqrt((bx * bx + by * by).mean()) / b0)
    return pl


def shock_3d(nx: int = 1024, ny: int = 128, nz: int = 128, ppc: int = 8,
             gamma_flow: float = 10.0, theta: float = 1e-4, r_p: float = 10.0,
             c: float = 0.45, seed: int = 1236) -> Plasma:
    """Periodic stand-in for the shock run of Sect. 4.2 in 3D3V: cold pair
    plasma streaming toward -x with Lorentz factor gamma_flow, no fields.
    Charge from Appendix A with <gamma> = gamma_flow; 4 binomial passes."""
    q_abs = charge_from_skin_depth(c, r_p, ppc, gamma_flow)
    beta = -math.sqrt(1.0 - 1.0 / gamma_flow**2)
    return uniform_plasma(3, nx, ny, nz, c, ppc, q_abs, theta, seed,
                          drift_axis=0, drift_beta_per_slot=np.full(ppc, beta),
                          meta=dict(workload="shock_3d3v_periodic", gamma_flow=gamma_flow,
                                    theta=theta, r_p=r_p, ppc=ppc, q_abs=q_abs,
                                    filter_passes=4))


def _relinearise(cell: np.ndarray, src: tuple, dst: tuple, shift_x: int) -> np.ndarray:
    """Cell indices of a (sx, sy, sz) block moved into a (nx, ny, nz) box at
    x offset shift_x."""
    c = cell.astype(np.int64)
    i, j, k = c % src[0], (c // src[0]) % src[1], c // (src[0] * src[1])
    return ((i + shift_x) + dst[0] * (j + dst[1] * k)).astype(np.int32)


def shock_tube(dim: int = 3, nx: int = 1024, ny: int = 128, nz: int = 128, ppc: int = 8,
               gamma_flow: float = 10.0, theta: float = 1e-4, r_p: float = 10.0,
               c: float = 0.45, wall: int = 2, x_inj: int = 512, x_max: float = 0.0,
               lt: int = 64, filter_passes: int = 4, seed: int = 1238) -> Plasma:
    """Shock set-up of Sect. 4.2: cold pair plasma streaming toward -x with
    Lorentz factor gamma_flow between a conducting wall at the node x = wall
    and a receding injector that starts at x = x_inj and moves at the speed of
    light (c cells per step) up to x_max (default nx - 3).  The injector lets
    in an upstream template: a block of lt cells (full y and z) of the same
    plasma, drawn independently and sorted by x (pairs stay co-located),
    advected at the bulk speed v_up = c beta.  Charge from Appendix A with
    <gamma> = gamma_flow.  meta["shock"] holds the boundary parameters and the
    template species (cells are indices of the lt x ny x nz block)."""
    if dim == 1:
        ny = nz = 1
    elif dim == 2:
        nz = 1
    x_max = float(x_max) if x_max > 0 else float(nx - 3)
    assert 1 <= wall < x_inj <= x_max <= nx - 3 and 2 * wall < nx
    q_abs = charge_from_skin_depth(c, r_p, ppc, gamma_flow)
    beta = math.sqrt(1.0 - 1.0 / gamma_flow**2)
    drift = np.full(ppc, -beta)
    fill = uniform_plasma(dim, x_inj - wall, ny, nz, c, ppc, q_abs, theta, seed,
                          drift_axis=0, drift_beta_per_slot=drift)
    for s in fill.species:
        s.cell = _relinearise(s.cell, (x_inj - wall, ny, nz), (nx, ny, nz), wall)
    tmpl = uniform_plasma(dim, lt, ny, nz, c, ppc, q_abs, theta, seed + 7919,
                          drift_axis=0, drift_beta_per_slot=drift)
    xt = (tmpl.species[0].cell.astype(np.int64) % lt).astype(np.float64) + \
        tmpl.species[0].off[0].astype(np.float64)
    order = np.argsort(xt, kind="stable")
    for s in tmpl.species:
        s.cell = np.ascontiguousarray(s.cell[order])
        s.off = np.ascontiguousarray(s.off[:, order])
        s.u = np.ascontiguousarray(s.u[:, order])
    fields = np.zeros((9, nz, ny, nx), dtype=np.float32)
    shock = dict(wall=int(wall), x_inj=float(x_inj), x_max=x_max, v_inj=float(c),
                 v_up=float(c * beta), lt=int(lt), templates=tmpl.species)
    return Plasma(dim=dim, nx=nx, ny=ny, nz=nz, c=c, species=fill.species, fields=fields,
                  meta=dict(workload=f"shock_{dim}d3v", gamma_flow=gamma_flow, theta=theta,
                            r_p=r_p, ppc=ppc, q_abs=q_abs, filter_passes=filter_passes,
                            shock=shock))


def injected_count(pl: Plasma, steps: int) -> int:
    """Upper bound on the particles per species that the injector of a
    shock_tube lets in over `steps` steps: the template density times the
    distance the injector front moves in template coordinates, plus one
    template block of slack for the partial blocks at both ends."""
    sh = pl.meta["shock"]
    nt = sh["templates"][0].n
    front = min(sh["x_inj"] + sh["v_inj"] * steps, sh["x_max"]) - sh["x_inj"] + sh["v_up"] * steps
    return int(math.ceil(front / sh["lt"] * nt)) + nt


def magnetic_modes(n: int, modes: int, seed: int) -> np.ndarray:
    """Perturbation fields of an n x n periodic box: for every wavenumber pair
    (m, k) in 1..modes, the lattice curl of
    A_z = (L / (2 pi |K|)) sin(2 pi m x / L + phi) sin(2 pi k y / L + psi)
    (|K| = sqrt(m^2 + k^2), seeded phases), so each field is discretely
    solenoidal with an amplitude of order 1.  float32 [modes^2, 3, 1, n, n],
    planes Bx (at (i, j+1/2)), By (at (i+1/2, j)), Bz (zero)."""
    gen = rng(seed)
    L = float(n)
    x = np.arange(n, dtype=np.float64)
    out = np.zeros((modes * modes, 3, 1, n, n), dtype=np.float32)
    for m in range(1, modes + 1):
        for k in range(1, modes + 1):
            phi, psi = 2.0 * math.pi * gen.random(2)
            K = math.sqrt(m * m + k * k)
            az = (L / (2.0 * math.pi * K)) * np.outer(np.sin(2.0 * math.pi * k * x / L + psi),
                                                      np.sin(2.0 * math.pi * m * x / L + phi))
            idx = (m - 1) * modes + (k - 1)
            out[idx, 0, 0] = np.roll(az, -1, axis=0) - az
            out[idx, 1, 0] = -(np.roll(az, -1, axis=1) - az)
    return out


def adjoint_box(n: int = 256, ppc: int = 32, theta: float = 0.1, sigma: float = 1.0,
                r_p: float = 4.0, modes: int = 8, db_over_b0: float = 0.1, c: float = 0.45,
                seed: int = 1239):
    """Differentiable turbulence-like set-up: a 2D3V periodic pair plasma at
    rest (Maxwell-Juettner theta) with the guide field B0 z-hat of
    magnetisation sigma (as in turbulence_2d) and an initial perturbation
    sum_m amps[m] * mode_m over modes^2 fields of magnetic_modes, with seeded
    amplitudes scaled so that the rms of dB is db_over_b0 * B0.  Returns
    (plasma without the perturbation, mode fields, amplitudes)."""
    mean_g = mj_mean_gamma(theta)
    q_abs = charge_from_skin_depth(c, r_p, ppc, mean_g)
    b0 = math.sqrt(sigma * ppc * q_abs * c * c * mean_g * 2.0)
    pl = uniform_plasma(2, n, n, 1, c, ppc, q_abs, theta, seed,
                        meta=dict(workload="adjoint_2d3v", theta=theta, sigma=sigma, r_p=r_p,
                                  ppc=ppc, q_abs=q_abs, b0=b0, mean_gamma=mean_g,
                                  filter_passes=0))
    pl.fields[5, 0] = np.float32(b0)
    mf = magnetic_modes(n, modes, seed + 100000)
    amps = rng(seed + 200000).normal(size=modes * modes)
    db = np.tensordot(amps, mf.astype(np.float64), axes=1)
    amps *= db_over_b0 * b0 / math.sqrt(float((db ** 2).sum(0).mean()))
    return pl, mf, amps.astype(np.float32)


def weibel_box(dim: int, n: int, ppc: int, gamma_b: float, theta: float, r_p: float = 10.0,
               c: float = 0.45, seed: int = 0) -> Plasma:
    """One Weibel box: 1D (n cells, beams along +-y as in weibel_1d) or 2D
    (n x n cells, beams along +-x in the plane, as in Sect. 4.1)."""
    if dim == 1:
        return weibel_1d(nx=n, ppc=ppc, gamma_b=gamma_b, theta=theta, r_p=r_p, c=c, seed=seed)
    q_abs = charge_from_skin_depth(c, r_p, ppc, gamma_b)
    beta_b = math.sqrt(1.0 - 1.0 / gamma_b**2)
    slots = np.where(np.arange(ppc) < ppc // 2, beta_b, -beta_b)
    return uniform_plasma(2, n, n, 1, c, ppc, q_abs, theta, seed, drift_axis=0,
                          drift_beta_per_slot=slots,
                          meta=dict(workload="weibel_2d3v", gamma_b=gamma_b, beta_b=beta_b,
                                    theta=theta, r_p=r_p, ppc=ppc, q_abs=q_abs,
                                    filter_passes=0))


def weibel_ensemble(count: int = 256, seed: int = 1237, max_1d: int = 4096, max_2d: int = 256):
    """Recipe of an ensemble of independent Weibel boxes with uneven sizes: half
    1D, half 2D; 1D lengths log-uniform in 128..max_1d, 2D sides log-uniform in
    32..max_2d, 16..128 particles per cell per species (even), gamma_b
    log-uniform in 1.5..10, theta log-uniform in 0.001..0.1.  Returns a list of
    (dim, n, ppc, gamma_b, theta, seed) tuples; weibel_box builds each."""
    gen = rng(seed)
    boxes = []
    for b in range(count):
        dim = 1 if gen.random() < 0.5 else 2
        lo, hi = (128, max_1d) if dim == 1 else (32, max_2d)
        n = int(round(math.exp(gen.uniform(math.log(lo), math.log(hi)))))
        ppc = 2 * int(round(math.exp(gen.uniform(math.log(16), math.log(128))) / 2))
        gamma_b = math.exp(gen.uniform(math.log(1.5), math.log(10.0)))
        theta = math.exp(gen.uniform(math.log(1e-3), math.log(0.1)))
        boxes.append((dim, n, ppc, gamma_b, theta, seed * 1000 + b))
    return boxes


CONFIGS = {
    "weibel_1d3v": weibel_1d,
    "turbulence_2d3v": turbulence_2d,
    "shock_3d3v_periodic": shock_3d,
}
