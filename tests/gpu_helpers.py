"""Helpers shared by the GPU parity tests: build the oracle state from the
GPU's (tile-sorted) particles so both sides hold particle i in slot i, and
compare with the tolerances the tests state."""
import numpy as np

import oracle

# Normwise relative tolerance on fields and energies per step for the FP32
# path against the FP64 oracle over short runs.
REL_TOL = 1e-5


def oracle_from_sim(sim):
    F, sp = sim.download()
    g = oracle.Grid(sim.dim, sim.nx, sim.ny, sim.nz, sim.c)
    osp = [oracle.Species(s["q"], s["m"], oracle.positions(g, s["cell"], s["off"]),
                          s["u"].astype(np.float64)) for s in sp]
    return g, F.astype(np.float64), osp, sp


def rel_err(a, ref):
    scale = np.abs(ref).max()
    return np.abs(np.asarray(a, dtype=np.float64) - ref).max() / max(scale, 1e-300)


def periodic_dx(g, xa, xb):
    """xa - xb on the periodic box, gridded rows only."""
    ext = np.array(g.extents(), dtype=np.float64)[:, None]
    d = np.asarray(xa[: g.dim], dtype=np.float64) - np.asarray(xb[: g.dim], dtype=np.float64)
    return d - np.round(d / ext) * ext


def current_scale(g, species):
    """c * sum_s |q_s| n_s / ncells: the current density of all particles
    streaming at c along one axis with the charges counted in absolute value.
    FP32 sums the per-particle ZigZag terms at this scale; when the species'
    currents cancel (co-moving pairs), the net field is far smaller than the
    terms and only this scale measures the rounding."""
    return g.c * sum(abs(s.q) * s.n for s in species) / g.ncells


def compare_fields(Fg, Fo, tol=REL_TOL, comps=range(9), floor=None):
    """Per component: max |GPU - oracle| <= tol * max(max |oracle|, floor[c])."""
    for c in comps:
        scale = np.abs(Fo[c]).max()
        if floor is not None:
            scale = max(scale, floor[c])
        if scale == 0.0:
            assert np.abs(Fg[c]).max() == 0.0, c
            continue
        e = np.abs(np.asarray(Fg[c], dtype=np.float64) - Fo[c]).max() / scale
        assert e < tol, (c, e, float(np.abs(Fo[c]).max()), scale)


def term_floor(g, terms):
    """Floors for compare_fields from the oracle's current-term magnitudes
    (oracle.step(..., terms=...): per step, the per-word sum of |ZigZag term|
    through the filter).  The scale is the largest such sum on any current
    word: FP32 sums the terms (not the net J, which cancels for co-moving
    pairs), rounds each to the fixed-point quantum of the shared-memory
    current, which is the same for every component, and follows a trajectory
    that drifts from the FP64 one by about 1e-6 of a cell within a few steps,
    so a word's error scales with the terms around it rather than with its own
    sum.  J holds the last step's deposit: that step's scale.  E adds -J every
    step: the sum of the steps' scales.  B, driven by c curl E: 2 D c times
    that."""
    acc = sum(float(t.max()) for t in terms)
    return [acc] * 3 + [2 * g.dim * g.c * acc] * 3 + [float(terms[-1].max())] * 3


def step_floor(g, species, k):
    """Floors for compare_fields after k steps: the E and J planes accumulate
    k current-scale terms, B is driven by c curl E over k steps."""
    j = current_scale(g, species)
    return [k * j] * 3 + [2 * g.dim * g.c * k * j] * 3 + [j] * 3


def compare_particles(g, spg, osp, xtol=2e-5, utol=1e-5):
    for s, o in zip(spg, osp):
        x = oracle.positions(g, s["cell"], s["off"])
        assert np.abs(periodic_dx(g, x, o.x)).max() < xtol
        du = np.abs(s["u"].astype(np.float64) - o.u)
        assert (du <= utol * np.maximum(1.0, np.abs(o.u))).all(), du.max()


def random_fields(shape, rs, amp_e=0.05, amp_b=0.3):
    """Smooth random periodic fields: a few low Fourier modes per component."""
    nz, ny, nx = shape
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    F = np.zeros((9,) + shape)
    for c in range(6):
        amp = amp_e if c < 3 else amp_b
        F[c] += amp * rs.normal()
        for _ in range(3):
            m = rs.integers(0, 3, size=3)
            ph = rs.uniform(0, 2 * np.pi)
            F[c] += amp * rs.normal() * np.cos(2 * np.pi * (m[0] * ii / nx + m[1] * jj / ny +
                                                             m[2] * kk / nz) + ph)
    return F.astype(np.float32)
