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
    """Per component: max |GPU - oracle| <= tol * max(max |oracle|, floor[c]).

    With a floor from term_floor (a dict), E and B take its global floors and
    J is compared cell by cell against that cell's own term magnitudes."""
    cell = None
    if isinstance(floor, dict):
        floor, cell = floor["floor"], floor["cell"]
    for c in comps:
        diff = np.abs(np.asarray(Fg[c], dtype=np.float64) - Fo[c])
        if cell is not None and c >= 6:
            scale = cell[c - 6]
            assert np.all(diff[scale == 0.0] == 0.0), c
            e = (diff / np.where(scale > 0.0, scale, 1.0)).max()
            assert e < tol, (c, e, float(np.abs(Fo[c]).max()), float(scale.max()))
            continue
        scale = np.abs(Fo[c]).max()
        if floor is not None:
            scale = max(scale, floor[c])
        if scale == 0.0:
            assert diff.max() == 0.0, c
            continue
        e = diff.max() / scale
        assert e < tol, (c, e, float(np.abs(Fo[c]).max()), scale)


# Per-cell J floors are not taken below this fraction of the largest cell's:
# the fixed-point shared-memory current rounds every term to a quantum of about
# 2^-19 |q| (current_quantum in the library), which a cell holding only a few
# small terms would see as a large relative error of its tiny term sum.
CELL_FLOOR_FRACTION = 1.0 / 16.0


def term_floor(g, terms):
    """Floors for compare_fields from the oracle's current-term magnitudes
    (oracle.step(..., terms=...): per step, the per-word sum of |ZigZag term|
    through the filter).  J, which holds the last step's deposit: per cell its
    own term sum, at least CELL_FLOOR_FRACTION of the largest.  E, which adds
    -J every step: the sum over steps of the largest term sum of its
    component.  B, driven by c curl E: 2 D c times the largest of those."""
    acc = sum(t.reshape(3, -1).max(axis=1) for t in terms)
    last = terms[-1]
    cell = [np.maximum(last[a], CELL_FLOOR_FRACTION * last[a].max()) for a in range(3)]
    return {"floor": [float(v) for v in acc] + [2 * g.dim * g.c * float(acc.max())] * 3 +
            [None] * 3, "cell": cell}


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
