"""FP64 CPU oracle of the relativistic PIC time step (arXiv:1906.06306).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  The product library
never loads it and shares no code with it.  The arithmetic lives in
``pic_oracle.c`` (plain C, double precision, periodic boxes or the shock
set-up's wall and injector); this module
compiles it with gcc on first use and marshals numpy arrays through ctypes.

Parity status of each function is pinned in ``tests/test_oracle_pins.py``:
Boris (closed-form gyration, E x B drift, pure-E kick), gather (exact for
constant and linear fields), ZigZag (hand sums from ``tests/golden`` and
discrete continuity), FDTD2 (Yee dispersion relation, div B), Binomial2
(Fourier response), whole step (Gauss law, energy, Weibel growth rate);
``tests/test_oracle_shock.py``: wall (specular reflection, charge continuity of
reflected particles, conductor standing waves) and injector (the box fills
with the advected upstream template, no gap and no duplicate);
``tests/test_oracle_adjoint.py``: the adjoint step (transpose identities and
central differences).  ``oracle.mutation_check`` plants 31 mistakes in copies
of the C sources and shows that each one fails a pin
(``tests/test_oracle_mutations.py``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic_oracle.c")
_SRC_ADJ = os.path.join(_HERE, "pic_oracle_adj.c")
_HDR = os.path.join(_HERE, "pic_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_D = ctypes.POINTER(ctypes.c_double)


class _Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("c", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile pic_oracle.c into liboracle.so (no fast-math, no FMA contraction)."""
    newest = max(os.path.getmtime(f) for f in (_SRC, _SRC_ADJ, _HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-shared", "-fPIC", _SRC, _SRC_ADJ, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    """The compiled oracle: liboracle.so built beside this file, or the library
    named by the ORACLE_LIB environment variable (a deliberately mutated build,
    used by ``oracle.mutation_check`` to show that the pins catch mistakes)."""
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(os.environ.get("ORACLE_LIB") or build())
        _lib.orc_kinetic_energy.restype = ctypes.c_double
        _lib.orc_inject.restype = ctypes.c_long
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


class Grid:
    """Periodic box: dim gridded dimensions, extents, Courant number c."""

    def __init__(self, dim, nx, ny=1, nz=1, c=0.45):
        self.dim, self.nx = int(dim), int(nx)
        self.ny = int(ny) if dim >= 2 else 1
        self.nz = int(nz) if dim >= 3 else 1
        self.c = float(c)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def ncells(self):
        return self.nx * self.ny * self.nz

    def extents(self):
        return (self.nx, self.ny, self.nz)[: self.dim]

    def c_struct(self):
        return ctypes.byref(_Grid(self.dim, self.nx, self.ny, self.nz, self.c))

    def zeros(self):
        return np.zeros((9,) + self.shape, dtype=np.float64)


class Species:
    """Oracle particles: x float64[3, n] absolute positions, u float64[3, n]."""

    def __init__(self, q, m, x, u):
        self.q, self.m = float(q), float(m)
        self.x = np.ascontiguousarray(x, dtype=np.float64)
        self.u = np.ascontiguousarray(u, dtype=np.float64)

    @property
    def n(self):
        return self.x.shape[1]


def positions(grid: Grid, cell: np.ndarray, off: np.ndarray) -> np.ndarray:
    """Absolute positions x = lattice index + offset, float64[3, n] (rows of
    non-gridded dimensions are 0), from the (cell, offset) particle layout."""
    cell = np.asarray(cell, dtype=np.int64)
    x = np.zeros((3, cell.shape[0]), dtype=np.float64)
    idx = [cell % grid.nx, (cell // grid.nx) % grid.ny, cell // (grid.nx * grid.ny)]
    for d in range(grid.dim):
        x[d] = idx[d].astype(np.float64) + np.asarray(off[d], dtype=np.float64)
    return x


def from_plasma(pl):
    """Grid, FP64 field planes and FP64 species from a workloads.Plasma; the
    FP32 bytes of the plasma are promoted exactly."""
    g = Grid(pl.dim, pl.nx, pl.ny, pl.nz, pl.c)
    F = pl.fields.astype(np.float64)
    sp = [Species(s.q, s.m, positions(g, s.cell, s.off), s.u.astype(np.float64))
          for s in pl.species]
    return g, F, sp


def push_half_b(g: Grid, F):
    lib().orc_push_half_b(g.c_struct(), _p(F))


def push_e(g: Grid, F):
    lib().orc_push_e(g.c_struct(), _p(F))


def add_cur(g: Grid, F):
    lib().orc_add_cur(g.c_struct(), _p(F))


def filter_binomial(g: Grid, F, passes: int):
    lib().orc_filter_binomial(g.c_struct(), _p(F), ctypes.c_int(passes))


def interp(g: Grid, F, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    e, b = np.zeros(3), np.zeros(3)
    lib().orc_interp(g.c_struct(), _p(F), _p(x), _p(e), _p(b))
    return e, b


def boris(u, e, b, qm: float, c: float):
    u = np.array(u, dtype=np.float64)
    lib().orc_boris(_p(u), _p(np.ascontiguousarray(e, dtype=np.float64)),
                    _p(np.ascontiguousarray(b, dtype=np.float64)), ctypes.c_double(qm), ctypes.c_double(c))
    return u


def higuera_cary(u, e, b, qm: float, c: float):
    u = np.array(u, dtype=np.float64)
    lib().orc_higuera_cary(_p(u), _p(np.ascontiguousarray(e, dtype=np.float64)),
                           _p(np.ascontiguousarray(b, dtype=np.float64)), ctypes.c_double(qm),
                           ctypes.c_double(c))
    return u


def set_field_order(order: int):
    """Spatial order of the field solver: 2 (FDTD2) or 4 (FDTD4)."""
    assert order in (2, 4)
    lib().orc_set_field_order(ctypes.c_int(order))


def set_pusher(name: str):
    """'boris' (Appendix C) or 'higuera_cary' for push_particles and step."""
    lib().orc_set_pusher(ctypes.c_int({"boris": 0, "higuera_cary": 1}[name]))


def zigzag(g: Grid, F, x1, x2, q: float):
    lib().orc_zigzag(g.c_struct(), _p(F), _p(np.ascontiguousarray(x1, dtype=np.float64)),
                     _p(np.ascontiguousarray(x2, dtype=np.float64)), ctypes.c_double(q))


def push_particles(g: Grid, F, sp: Species):
    """interp_em + push for one species; returns (x_old, dx)."""
    x_old = np.zeros((3, sp.n))
    dx = np.zeros((3, sp.n))
    lib().orc_push_particles(g.c_struct(), _p(F), _p(sp.x), _p(sp.u), ctypes.c_long(sp.n),
                             ctypes.c_double(sp.q / sp.m), _p(x_old), _p(dx))
    return x_old, dx


def deposit(g: Grid, F, x_old, dx, q: float):
    lib().orc_deposit(g.c_struct(), _p(F), _p(x_old), _p(dx), ctypes.c_long(x_old.shape[1]),
                      ctypes.c_double(q))


def deposit_abs(g: Grid, F, x_old, dx, q: float):
    """deposit() with every ZigZag term added as its absolute value: per
    current word, the sum of |contribution| over the moves (it bounds |J| and
    equals it for a single move)."""
    lib().orc_deposit_abs(g.c_struct(), _p(F), _p(x_old), _p(dx), ctypes.c_long(x_old.shape[1]),
                          ctypes.c_double(q))


def step(g: Grid, F, species, passes: int = 0, nsteps: int = 1, terms=None):
    """`nsteps` full time steps in the order of Table 1 (in place).  With a
    list `terms`, each step appends the 3 planes of its current's term
    magnitudes: deposit_abs of the step's moves, through the same filter
    passes (whose weights are positive, so the planes still bound |J|)."""
    ns = len(species)
    xs = (_D * ns)(*[_p(s.x) for s in species])
    us = (_D * ns)(*[_p(s.u) for s in species])
    n = (ctypes.c_long * ns)(*[s.n for s in species])
    q = (ctypes.c_double * ns)(*[s.q for s in species])
    m = (ctypes.c_double * ns)(*[s.m for s in species])
    work = np.zeros(6 * sum(s.n for s in species))
    for _ in range(nsteps):
        lib().orc_step(g.c_struct(), _p(F), xs, us, n, q, m, ctypes.c_int(ns),
                       ctypes.c_int(passes), _p(work))
        if terms is not None:  # the step's moves are left in `work`: x_old, then dx
            A = g.zeros()
            o = 0
            for s in species:
                x_old = np.ascontiguousarray(work[o:o + 3 * s.n].reshape(3, s.n))
                dx = np.ascontiguousarray(work[o + 3 * s.n:o + 6 * s.n].reshape(3, s.n))
                deposit_abs(g, A, x_old, dx, s.q)
                o += 6 * s.n
            filter_binomial(g, A, passes)
            terms.append(A[6:9].copy())


def set_wall(w: int, i_zero: int = 0):
    """Conducting wall on the node plane x = w (0: none) for push_particles,
    deposit and step, with E and B zeroed at i >= i_zero after each field
    update of step (Sect. 4.2 shock set-up)."""
    lib().orc_set_wall(ctypes.c_long(w), ctypes.c_long(i_zero))


def wall_fields(g: Grid, F, w: int, i_zero: int):
    lib().orc_wall_fields(g.c_struct(), _p(F), ctypes.c_long(w), ctypes.c_long(i_zero))


class Injector:
    """Receding injector of the shock set-up (Sect. 4.2): `templates` is one
    (x float64[3, nt], u float64[3, nt]) upstream block per species, x in
    [0, lt) x ny x nz and sorted by x; it is repeated along x and advected at
    -v_up, and the injector X(s) = min(x0 + v_inj s, x_max) lets in, during
    step s, the template particles that cross it."""

    def __init__(self, templates, lt, x0, x_max, v_inj, v_up):
        self.templates = [(np.ascontiguousarray(x, dtype=np.float64),
                           np.ascontiguousarray(u, dtype=np.float64)) for x, u in templates]
        self.lt, self.x0, self.x_max = int(lt), float(x0), float(x_max)
        self.v_inj, self.v_up = float(v_inj), float(v_up)

    def inject(self, s: int, species):
        """Append the particles entering during step s to each species."""
        counts = []
        for (xt, ut), sp in zip(self.templates, species):
            nt = xt.shape[1]
            cap = nt * (2 + int(np.ceil((self.v_inj + self.v_up) / self.lt))) + 16
            xo, uo = np.zeros((3, cap)), np.zeros((3, cap))
            k = lib().orc_inject(_p(xt), _p(ut), ctypes.c_long(nt), ctypes.c_long(self.lt),
                                 ctypes.c_double(self.x0), ctypes.c_double(self.x_max),
                                 ctypes.c_double(self.v_inj), ctypes.c_double(self.v_up),
                                 ctypes.c_long(s), _p(xo), _p(uo), ctypes.c_long(cap))
            assert k >= 0
            sp.x = np.ascontiguousarray(np.concatenate([sp.x, xo[:, :k]], axis=1))
            sp.u = np.ascontiguousarray(np.concatenate([sp.u, uo[:, :k]], axis=1))
            counts.append(int(k))
        return counts


def shock_from_plasma(pl):
    """(wall, i_zero, Injector) of a workloads.shock_tube plasma; i_zero is the
    first lattice index past the injector's last position plus one cell."""
    sh = pl.meta["shock"]
    tg = Grid(pl.dim, sh["lt"], pl.ny, pl.nz, pl.c)
    temps = [(positions(tg, t.cell, t.off), t.u.astype(np.float64)) for t in sh["templates"]]
    inj = Injector(temps, sh["lt"], sh["x_inj"], sh["x_max"], sh["v_inj"], sh["v_up"])
    return sh["wall"], int(np.floor(sh["x_max"])) + 2, inj


def step_shock(g: Grid, F, species, injector, s0: int, passes: int = 0, nsteps: int = 1,
               terms=None):
    """`nsteps` steps of the shock set-up from step index s0: each a full step
    (with the wall set by set_wall) followed by the injection of that step;
    `terms` as in step()."""
    for t in range(nsteps):
        step(g, F, species, passes=passes, nsteps=1, terms=terms)
        if injector is not None:
            injector.inject(s0 + t, species)


def adj_step(g: Grid, F, species, xbar, ubar, A, passes: int = 0):
    """Reverse of one `step` (FDTD2, Boris): F and species are the forward
    state at the start of the step; A (adjoint field planes), xbar[s]
    (float64[3, n]) and ubar[s] (float64[3, n]) go in as the gradient with
    respect to the state after the step and come out with respect to the
    state before it."""
    ns = len(species)
    xs = (_D * ns)(*[_p(s.x) for s in species])
    us = (_D * ns)(*[_p(s.u) for s in species])
    n = (ctypes.c_long * ns)(*[s.n for s in species])
    q = (ctypes.c_double * ns)(*[s.q for s in species])
    m = (ctypes.c_double * ns)(*[s.m for s in species])
    xb = (_D * ns)(*[_p(a) for a in xbar])
    ub = (_D * ns)(*[_p(a) for a in ubar])
    work = np.zeros(9 * g.ncells)
    lib().orc_adj_step(g.c_struct(), _p(F), xs, us, n, q, m, ctypes.c_int(ns), ctypes.c_int(passes),
                       xb, ub, _p(A), _p(work))


def gradient(g: Grid, F, species, nsteps: int, loss_grad, passes: int = 0):
    """Gradient of a loss of the state after `nsteps` steps with respect to
    the initial state, by the discrete adjoint: the forward states are kept
    (small cases), then adj_step runs backwards.  loss_grad(F, species) returns
    (A, xbar, ubar) for the final state.  Returns (A, xbar, ubar) at t = 0;
    F and species are left at the final state."""
    states = []
    for _ in range(nsteps):
        states.append((F.copy(), [Species(s.q, s.m, s.x.copy(), s.u.copy()) for s in species]))
        step(g, F, species, passes=passes)
    A, xbar, ubar = loss_grad(F, species)
    for Fs, sps in reversed(states):
        adj_step(g, Fs, sps, xbar, ubar, A, passes=passes)
    return A, xbar, ubar


def charge_density(g: Grid, species):
    rho = np.zeros(g.shape)
    for s in species:
        lib().orc_charge_density(g.c_struct(), _p(s.x), ctypes.c_long(s.n),
                                 ctypes.c_double(s.q), _p(rho))
    return rho


def div_e(g: Grid, F):
    out = np.zeros(g.shape)
    lib().orc_div_e(g.c_struct(), _p(F), _p(out))
    return out


def div_b(g: Grid, F):
    out = np.zeros(g.shape)
    lib().orc_div_b(g.c_struct(), _p(F), _p(out))
    return out


def field_energy(g: Grid, F):
    out = np.zeros(2)
    lib().orc_field_energy(g.c_struct(), _p(F), _p(out))
    return float(out[0]), float(out[1])


def kinetic_energy(g: Grid, sp: Species):
    return float(lib().orc_kinetic_energy(_p(sp.u), ctypes.c_long(sp.n), ctypes.c_double(sp.m),
                                          ctypes.c_double(g.c)))


def energies(g: Grid, F, species):
    """[0.5 sum E^2, 0.5 sum B^2, kinetic energy of each species]."""
    ee, eb = field_energy(g, F)
    return [ee, eb] + [kinetic_energy(g, s) for s in species]


def gauss_residual(g: Grid, F, species, passes: int = 0):
    """div E - F^p(rho) on the nodes.  The Binomial2 filter is linear and
    translation invariant, so it commutes with the divergence; with p passes
    on J every step this residual is conserved by the scheme."""
    rho = charge_density(g, species)
    if passes:
        tmp = g.zeros()
        tmp[6] = rho
        filter_binomial(g, tmp, passes)
        rho = tmp[6]
    return div_e(g, F) - rho


def tile_keys(cell: np.ndarray, nx: int, ny: int, nz: int, tile) -> np.ndarray:
    """Tile index of each particle for tiles of tile = (tx, ty, tz) cells, tiles
    numbered x-fastest: the definition of the sorted particle layout."""
    cell = np.asarray(cell, dtype=np.int64)
    i, j, k = cell % nx, (cell // nx) % ny, cell // (nx * ny)
    ntx = -(-nx // tile[0])
    nty = -(-ny // tile[1])
    return (i // tile[0]) + ntx * ((j // tile[1]) + nty * (k // tile[2]))


def tile_sort_reference(cell, nx, ny, nz, tile):
    """Stable permutation by tile key and the tile start offsets (length
    ntiles + 1): a plain stable sort and a histogram."""
    key = tile_keys(cell, nx, ny, nz, tile)
    ntiles = (-(-nx // tile[0])) * (-(-ny // tile[1])) * (-(-nz // tile[2]))
    perm = np.argsort(key, kind="stable")
    start = np.zeros(ntiles + 1, dtype=np.int64)
    start[1:] = np.cumsum(np.bincount(key, minlength=ntiles))
    return perm, start
