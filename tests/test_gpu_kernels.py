"""Kernel-level parity of the CUDA path (through the C ABI) with the FP64
oracle: FDTD2 updates, Binomial2 filter, gather + Boris + move, ZigZag deposit
and the tile sort.  Sizes span several tiles with ragged edges."""
import numpy as np
import pytest

import oracle
import workloads

from gpu_helpers import (compare_fields, compare_particles, oracle_from_sim, periodic_dx,
                         random_fields, rel_err)

pytestmark = pytest.mark.gpu

SHAPES = {1: (37, 1, 1), 2: (29, 23, 1), 3: (13, 11, 9)}


def _sim(dim, shape, fields, species, **tun):
    from paper_1906_06306_gb300 import Simulation

    nx, ny, nz = shape
    return Simulation(dim, nx, ny, nz, 0.45, fields, species, tuning=tun or None)


def _empty_species(dim):
    return [dict(q=-1.0, m=1.0, cell=np.zeros(0, np.int32), off=np.zeros((dim, 0), np.float32),
                 u=np.zeros((3, 0), np.float32))]


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_field_updates_match_oracle(dim):
    from paper_1906_06306_gb300 import PIC_FIELD_B_HALF, PIC_FIELD_E

    nx, ny, nz = SHAPES[dim]
    rs = np.random.default_rng(100 + dim)
    F32 = random_fields((nz, ny, nx), rs)
    F32[6:9] = (0.01 * rs.normal(size=(3, nz, ny, nx))).astype(np.float32)
    sim = _sim(dim, SHAPES[dim], F32, _empty_species(dim))
    g = oracle.Grid(dim, nx, ny, nz, 0.45)
    F = F32.astype(np.float64)
    sim.field_update(PIC_FIELD_B_HALF)
    oracle.push_half_b(g, F)
    compare_fields(sim.download()[0], F, tol=1e-6)
    sim.field_update(PIC_FIELD_E)
    oracle.push_e(g, F)
    oracle.add_cur(g, F)
    compare_fields(sim.download()[0], F, tol=1e-6)
    sim.close()


@pytest.mark.parametrize("dim,shape", [(1, (64, 1, 1)), (2, (32, 20, 1)), (2, (4, 3, 1)),
                                       (3, (16, 12, 8)), (3, (8, 5, 3))])
def test_field_updates_four_points_per_thread_match_oracle(dim, shape):
    """Rows whose length is a multiple of 4 take the FDTD2 kernels with four
    x points per thread (16-byte loads and stores, wrapped x neighbours at
    both row ends), down to a row of one quad."""
    from paper_1906_06306_gb300 import PIC_FIELD_B_HALF, PIC_FIELD_E

    nx, ny, nz = shape
    rs = np.random.default_rng(110 + nx + ny + nz)
    F32 = random_fields((nz, ny, nx), rs)
    F32[6:9] = (0.01 * rs.normal(size=(3, nz, ny, nx))).astype(np.float32)
    sim = _sim(dim, shape, F32, _empty_species(dim))
    g = oracle.Grid(dim, nx, ny, nz, 0.45)
    F = F32.astype(np.float64)
    for _ in range(3):
        sim.field_update(PIC_FIELD_B_HALF)
        oracle.push_half_b(g, F)
        compare_fields(sim.download()[0], F, tol=1e-6)
        sim.field_update(PIC_FIELD_E)
        oracle.push_e(g, F)
        oracle.add_cur(g, F)
        compare_fields(sim.download()[0], F, tol=1e-6)
    sim.close()


@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("passes", [1, 2, 3])
def test_binomial_filter_matches_oracle(dim, passes):
    nx, ny, nz = SHAPES[dim]
    rs = np.random.default_rng(200 + dim)
    F32 = np.zeros((9, nz, ny, nx), np.float32)
    F32[6:9] = rs.normal(size=(3, nz, ny, nx)).astype(np.float32)
    sim = _sim(dim, SHAPES[dim], F32, _empty_species(dim))
    g = oracle.Grid(dim, nx, ny, nz, 0.45)
    F = F32.astype(np.float64)
    sim.filter_current(passes)
    oracle.filter_binomial(g, F, passes)
    compare_fields(sim.download()[0], F, tol=1e-6)
    sim.close()


@pytest.mark.parametrize("shape", [(37, 11, 9), (68, 19, 41), (4, 8, 2), (1, 1, 3), (2, 3, 1),
                                   (1024, 256, 40), (132, 20, 6)])
def test_binomial_filter_3d_z_runs_match_oracle(shape):
    """The 3D pass marches along z over (x, y) columns of 128 x 16 points: rows
    whose x extent is not a multiple of 4 (4-byte copies only), ragged columns
    (68; 132 = 128 + 4, whose bulk row copies are 4 points long), several z
    runs with a ragged last one, extents below the column and the halo, and a
    box of many columns whose runs span all its planes (1024 x 256 x 40)."""
    nx, ny, nz = shape
    rs = np.random.default_rng(sum(shape))
    F32 = np.zeros((9, nz, ny, nx), np.float32)
    F32[6:9] = rs.normal(size=(3, nz, ny, nx)).astype(np.float32)
    sim = _sim(3, shape, F32, _empty_species(3))
    g = oracle.Grid(3, nx, ny, nz, 0.45)
    F = F32.astype(np.float64)
    sim.filter_current(3)
    oracle.filter_binomial(g, F, 3)
    compare_fields(sim.download()[0], F, tol=1e-6, comps=range(6, 9))
    sim.close()


@pytest.mark.parametrize("shape", [(29, 23), (1030, 7), (4, 8), (1, 3), (2, 1), (2048, 64),
                                   (1024, 1024), (1036, 9)])
def test_binomial_filter_2d_y_runs_match_oracle(shape):
    """The 2D pass marches along y over 1024-point x columns: ragged columns
    (1030; 1036 = 1024 + 12, whose bulk row copies are 12 points long; 2048 +
    halo), rows whose x extent is not a multiple of 4 (4-byte copies only),
    extents below the halo, and the 1024^2 plane of the turbulence box."""
    nx, ny = shape
    rs = np.random.default_rng(nx + 7 * ny)
    F32 = np.zeros((9, 1, ny, nx), np.float32)
    F32[6:9] = rs.normal(size=(3, 1, ny, nx)).astype(np.float32)
    sim = _sim(2, (nx, ny, 1), F32, _empty_species(2))
    g = oracle.Grid(2, nx, ny, 1, 0.45)
    F = F32.astype(np.float64)
    sim.filter_current(3)
    oracle.filter_binomial(g, F, 3)
    compare_fields(sim.download()[0], F, tol=1e-6, comps=range(6, 9))
    sim.close()


def _plasma(dim, shape, ppc, theta, seed):
    nx, ny, nz = shape
    return workloads.uniform_plasma(dim, nx, ny, nz, 0.45, ppc, 0.02, theta, seed)


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_gather_push_matches_oracle_and_move_replays_bit_exact(dim):
    nx, ny, nz = SHAPES[dim]
    pl = _plasma(dim, SHAPES[dim], 6, 0.5, 300 + dim)
    pl.fields[:] = random_fields((nz, ny, nx), np.random.default_rng(301))
    from paper_1906_06306_gb300 import Simulation

    sim = Simulation.from_plasma(pl, tuning=dict(sort_every=1000))
    g, F, osp, sp0 = oracle_from_sim(sim)
    sim.gather_push()
    sim.check()
    _, spg = sim.download()
    for o in osp:
        oracle.push_particles(g, F, o)
    compare_particles(g, spg, osp, xtol=2e-6, utol=2e-6)
    # cell bookkeeping: replay the documented FP32 position update on the CPU
    f32 = np.float32
    c = f32(0.45)
    for s0, s1 in zip(sp0, spg):
        u = s1["u"]
        g2 = ((f32(1) + u[0] * u[0]) + u[1] * u[1]) + u[2] * u[2]
        r = f32(1) / np.sqrt(g2, dtype=f32)
        idx = [s0["cell"] % nx, (s0["cell"] // nx) % ny, s0["cell"] // (nx * ny)]
        for d in range(dim):
            dn = (c * u[d]) * r
            o = s0["off"][d] + dn
            k = np.zeros_like(s0["cell"])
            lo, hi = o < 0, o >= 1
            o = np.where(lo, o + f32(1), np.where(hi, o - f32(1), o)).astype(f32)
            k[lo], k[hi] = -1, 1
            edge = lo & (o >= 1)
            o[edge], k[edge] = 0, 0
            assert np.array_equal(o.view(np.int32), s1["off"][d].view(np.int32))
            idx[d] = (idx[d] + k) % (nx, ny, nz)[d]
        assert np.array_equal(idx[0] + nx * (idx[1] + ny * idx[2]), s1["cell"])
    sim.close()


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_deposit_matches_oracle_zigzag_of_the_same_moves(dim):
    """J of pic_deposit equals the oracle's ZigZag current of the moves the GPU
    made (old position, new position, out-of-plane displacement c u / gamma)."""
    nx, ny, nz = SHAPES[dim]
    pl = _plasma(dim, SHAPES[dim], 8, 1.0, 400 + dim)
    pl.fields[:] = random_fields((nz, ny, nx), np.random.default_rng(401))
    from paper_1906_06306_gb300 import Simulation

    sim = Simulation.from_plasma(pl, tuning=dict(sort_every=1000))
    g, F, osp, sp0 = oracle_from_sim(sim)
    sim.gather_push()
    sim.deposit()
    sim.check()
    Fg, spg = sim.download()
    Fo = np.zeros_like(F)
    for s0, s1 in zip(sp0, spg):
        x_old = oracle.positions(g, s0["cell"], s0["off"])
        x_new = oracle.positions(g, s1["cell"], s1["off"])
        dx = np.zeros_like(x_old)
        dx[:dim] = periodic_dx(g, x_new, x_old)
        u = s1["u"].astype(np.float64)
        gam = np.sqrt(1.0 + (u * u).sum(axis=0))
        dx[dim:] = 0.45 * u[dim:] / gam
        oracle.deposit(g, Fo, np.ascontiguousarray(x_old), np.ascontiguousarray(dx), s0["q"])
    for c in range(6, 9):
        assert rel_err(Fg[c], Fo[c]) < 1e-5, c
    sim.close()


@pytest.mark.parametrize("dim,tile", [(1, (8,)), (2, (8, 4)), (3, (4, 4, 2))])
def test_sort_groups_particles_by_tile(dim, tile):
    nx, ny, nz = SHAPES[dim]
    pl = _plasma(dim, SHAPES[dim], 5, 0.3, 500 + dim)
    rs = np.random.default_rng(501)
    for s in pl.species:  # scramble the input order
        p = rs.permutation(s.n)
        s.cell, s.off, s.u = s.cell[p].copy(), s.off[:, p].copy(), s.u[:, p].copy()
    from paper_1906_06306_gb300 import Simulation

    sim = Simulation.from_plasma(pl, tuning=dict(tile=list(tile) + [1] * (3 - dim)))
    _, spg = sim.download()
    t3 = tuple(tile) + (1,) * (3 - dim)
    for s_in, s_out in zip(pl.species, spg):
        key_out = oracle.tile_keys(s_out["cell"], nx, ny, nz, t3)
        _, start = oracle.tile_sort_reference(s_in.cell, nx, ny, nz, t3)
        # bit-exact grouping: the key sequence is the sorted key sequence
        assert np.array_equal(key_out, np.sort(oracle.tile_keys(s_in.cell, nx, ny, nz, t3)))
        assert np.array_equal(np.searchsorted(key_out, np.arange(len(start) - 1)), start[:-1])
        # same particles (bytes) in every tile
        def rows(s):
            return np.concatenate([s["cell"][None].view(np.float32), s["off"], s["u"]]).T.copy()
        a = rows(s_out)
        b = rows(dict(cell=s_in.cell, off=s_in.off, u=s_in.u))
        for t in range(len(start) - 1):
            sa = a[start[t]:start[t + 1]].view(np.int32)
            kb = oracle.tile_keys(s_in.cell, nx, ny, nz, t3) == t
            sb = b[kb].view(np.int32)
            assert np.array_equal(np.unique(sa, axis=0), np.unique(sb, axis=0))
    sim.close()


def test_sort_orders_3d_tiles_by_sub_tile():
    """3D tiles of 8x8x4 cells are sorted into 4x4x2 sub-tile bins, tile-major
    (sub-tile x fastest): the bin sequence of the output is the sorted bin
    sequence of the input, ragged last tiles included, and every bin holds
    the same particles (bytes)."""
    nx, ny, nz = 21, 18, 10
    pl = _plasma(3, (nx, ny, nz), 3, 0.3, 509)
    rs = np.random.default_rng(510)
    for s in pl.species:  # scramble the input order
        p = rs.permutation(s.n)
        s.cell, s.off, s.u = s.cell[p].copy(), s.off[:, p].copy(), s.u[:, p].copy()
    from paper_1906_06306_gb300 import Simulation

    sim = Simulation.from_plasma(pl, tuning=dict(tile=[8, 8, 4]))
    _, spg = sim.download()
    T, S = (8, 8, 4), (4, 4, 2)

    def bins(cell):
        cell = np.asarray(cell, dtype=np.int64)
        i, j, k = cell % nx, (cell // nx) % ny, cell // (nx * ny)
        tile = oracle.tile_keys(cell, nx, ny, nz, T)
        ns = [-(-t // u) for t, u in zip(T, S)]
        sub = ((i % T[0]) // S[0]) + ns[0] * (((j % T[1]) // S[1]) + ns[1] * ((k % T[2]) // S[2]))
        return tile * (ns[0] * ns[1] * ns[2]) + sub

    for s_in, s_out in zip(pl.species, spg):
        b_out, b_in = bins(s_out["cell"]), bins(s_in.cell)
        assert np.array_equal(b_out, np.sort(b_in))

        def rows(cell, off, u):
            return np.concatenate([np.asarray(cell)[None].view(np.float32), off, u]).T.copy()

        a = rows(s_out["cell"], s_out["off"], s_out["u"]).view(np.int32)
        b = rows(s_in.cell, s_in.off, s_in.u).view(np.int32)
        for key in np.unique(b_in):
            assert np.array_equal(np.unique(a[b_out == key], axis=0), np.unique(b[b_in == key], axis=0))
    sim.close()


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_higuera_cary_gather_push_matches_oracle(dim):
    nx, ny, nz = SHAPES[dim]
    pl = _plasma(dim, SHAPES[dim], 6, 2.0, 600 + dim)
    pl.fields[:] = random_fields((nz, ny, nx), np.random.default_rng(601), amp_e=0.1, amp_b=0.6)
    from paper_1906_06306_gb300 import Simulation

    sim = Simulation.from_plasma(pl, tuning=dict(sort_every=1000))
    sim.set_pusher("higuera_cary")
    g, F, osp, _ = oracle_from_sim(sim)
    sim.gather_push()
    sim.check()
    _, spg = sim.download()
    oracle.set_pusher("higuera_cary")
    try:
        for o in osp:
            oracle.push_particles(g, F, o)
    finally:
        oracle.set_pusher("boris")
    compare_particles(g, spg, osp, xtol=2e-6, utol=2e-6)
    sim.close()


def test_higuera_cary_keeps_exb_drift_on_gpu():
    """Uniform E = beta B y-hat, B z-hat: particles moving with the drift
    velocity beta x-hat (gamma = 7.1) keep it over 300 steps in FP32."""
    from paper_1906_06306_gb300 import Simulation

    nx, ny = 16, 8
    beta, bz = 0.99, 0.3
    gam = 1.0 / np.sqrt(1.0 - beta**2)
    n = 64
    rs = np.random.default_rng(602)
    fields = np.zeros((9, 1, ny, nx), np.float32)
    fields[1] = beta * bz
    fields[5] = bz
    u = np.zeros((3, n), np.float32)
    u[0] = gam * beta
    sp = [dict(q=q, m=1.0, cell=rs.integers(0, nx * ny, n).astype(np.int32),
               off=rs.random((2, n)).astype(np.float32), u=u.copy()) for q in (1e-9, -1e-9)]
    sim = Simulation(2, nx, ny, 1, 0.45, fields, sp, tuning=dict(sort_every=1000))
    sim.set_pusher("higuera_cary")
    for _ in range(300):
        sim.gather_push()  # fields stay uniform: no deposit, no field update
    sim.check()
    _, spg = sim.download()
    for s in spg:
        assert np.abs(s["u"][0] - gam * beta).max() < 2e-5 * gam
        assert np.abs(s["u"][1:]).max() < 2e-5 * gam
    sim.close()


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_fdtd4_field_updates_match_oracle(dim):
    from paper_1906_06306_gb300 import PIC_FIELD_B_HALF, PIC_FIELD_E

    nx, ny, nz = SHAPES[dim]
    rs = np.random.default_rng(700 + dim)
    F32 = random_fields((nz, ny, nx), rs)
    F32[6:9] = (0.01 * rs.normal(size=(3, nz, ny, nx))).astype(np.float32)
    sim = _sim(dim, SHAPES[dim], F32, _empty_species(dim))
    sim.set_field_solver(4)
    g = oracle.Grid(dim, nx, ny, nz, 0.45)
    F = F32.astype(np.float64)
    oracle.set_field_order(4)
    try:
        sim.field_update(PIC_FIELD_B_HALF)
        oracle.push_half_b(g, F)
        compare_fields(sim.download()[0], F, tol=1e-6)
        sim.field_update(PIC_FIELD_E)
        oracle.push_e(g, F)
        oracle.add_cur(g, F)
        compare_fields(sim.download()[0], F, tol=1e-6)
    finally:
        oracle.set_field_order(2)
    sim.close()
