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


def compare_fields(Fg, Fo, tol=REL_TOL, comps=range(9)):
    for c in comps:
        if np.abs(Fo[c]).max() == 0.0:
            assert np.abs(Fg[c]).max() == 0.0, c
            continue
        e = rel_err(Fg[c], Fo[c])
        assert e < tol, (c, e)


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
