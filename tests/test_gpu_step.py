"""Whole-step parity of pic_step (fused gather + push + deposit, field updates,
filter) with the FP64 oracle, plus edge cases and invariants."""
import math

import numpy as np
import pytest

import oracle
import workloads

from gpu_helpers import (REL_TOL, compare_fields, compare_particles, oracle_from_sim,
                         periodic_dx, rel_err, term_floor)

pytestmark = pytest.mark.gpu


def _small_configs():
    return {
        "weibel_1d": (workloads.weibel_1d(nx=200, ppc=16, seed=21), 0, {}),
        "turb_2d": (workloads.turbulence_2d(n=40, ppc=4, r_p=4.0, theta=0.3, sigma=10.0,
                                            modes=4, seed=22), 0, dict(tile=[16, 16, 1])),
        "shock_3d": (workloads.shock_3d(nx=20, ny=12, nz=10, ppc=2, seed=23), 2,
                     dict(tile=[8, 8, 4])),
        "turb_2d_filtered": (workloads.turbulence_2d(n=36, ppc=4, r_p=4.0, theta=0.3, sigma=1.0,
                                                     modes=4, seed=24), 3, dict(tile=[8, 8, 1])),
    }


@pytest.mark.parametrize("name", list(_small_configs()))
def test_step_matches_oracle_over_short_run(name):
    from paper_1906_06306_gb300 import Simulation

    pl, passes, tun = _small_configs()[name]
    sim = Simulation.from_plasma(pl, tuning=dict(tun, sort_every=1000, filter_passes=passes))
    g, F, osp, _ = oracle_from_sim(sim)
    terms = []
    for k in range(1, 9):
        sim.step(1)
        oracle.step(g, F, osp, passes=passes, terms=terms)
        Fg, spg = sim.download()
        compare_fields(Fg, F, floor=term_floor(g, terms))
        compare_particles(g, spg, osp)
    sim.check()
    en = sim.energies()
    ref = oracle.energies(g, F, osp)
    # field energies that are a negligible part of the total (cancelled
    # currents of co-moving pairs) are compared at 1e-6 of the total energy
    total = sum(ref)
    for a, b in zip(en[:2 + len(osp)], ref):
        assert abs(a - b) <= REL_TOL * max(abs(b), 1e-6 * total), (a, b, total)
    sim.close()


@pytest.mark.parametrize("tile,halo,aligned", [((16, 8), 3, True), ((16, 16), 3, True),
                                               ((16, 8), 2, True), ((16, 8), 3, False),
                                               ((16, 8), 2, False)])
def test_fixed_and_generic_window_kernels_match_oracle(tile, halo, aligned):
    """The 2D particle kernel has compile-time window instantiations for the
    windows of 16x8 and 16x16 tiles with halo 3; each of them and the generic
    kernel (halo 2) against the oracle on a box that spans several tiles with
    ragged edges, with sorts and strays.  Rows of a multiple of 4 particles
    stream the records with bulk copies; rows of another length (one spare
    slot) take the plain loads."""
    from paper_1906_06306_gb300 import Simulation

    pl = workloads.turbulence_2d(n=52, ppc=4, r_p=4.0, theta=0.3, sigma=10.0, modes=4, seed=26)
    cap = None if aligned else [s.n + 1 for s in pl.species]
    sim = Simulation.from_plasma(pl, tuning=dict(tile=[tile[0], tile[1], 1], halo=halo,
                                                 sort_every=1000),
                                 capacity=cap, align_rows=aligned)
    g, F, osp, _ = oracle_from_sim(sim)
    terms = []
    for k in range(1, 7):
        sim.step(1)
        oracle.step(g, F, osp, terms=terms)
    Fg, spg = sim.download()
    compare_fields(Fg, F, floor=term_floor(g, terms))
    compare_particles(g, spg, osp)
    sim.close()


def test_step_with_frequent_sorts_and_strays_matches_oracle_fields():
    """A hot plasma, halo 1 and a sort every 5 steps: many particles leave
    their tile window between sorts and take the global-memory path; the
    fields still follow the oracle (particle order differs, fields do not)."""
    from paper_1906_06306_gb300 import Simulation

    pl = workloads.uniform_plasma(2, 34, 30, 1, 0.45, 4, 0.01, 2.0, seed=25)
    sim = Simulation.from_plasma(pl, tuning=dict(tile=[8, 8, 1], halo=1, sort_every=5))
    g, F, osp, _ = oracle_from_sim(sim)
    terms = []
    for _ in range(20):
        sim.step(1)
        oracle.step(g, F, osp, terms=terms)
    Fg, spg = sim.download()
    compare_fields(Fg, F, floor=term_floor(g, terms))
    # same particles, in another order: compare sorted kinetic energies
    for s, o in zip(spg, osp):
        ug = np.sort((s["u"].astype(np.float64) ** 2).sum(0))
        uo = np.sort((o.u ** 2).sum(0))
        assert np.abs(ug - uo).max() < 1e-4 * max(1.0, uo.max())
    sim.check()
    sim.close()


def test_strays_beyond_the_queue_are_run_by_their_lanes():
    """A plasma drifting at 0.99 c along x, 4x4 tiles with halo 1 (a particle
    strays as soon as it leaves its tile) and no sort: after a few steps most
    of a block's ~680 particles per species stray, more than the stray queue
    holds, so lanes that find it full run their particle through global memory
    at once.  Fields and particles follow the oracle slot by slot."""
    from paper_1906_06306_gb300 import binding as B
    from paper_1906_06306_gb300 import Simulation

    ppc = 128
    pl = workloads.uniform_plasma(2, 64, 64, 1, 0.45, ppc, 1e-4, 0.01, seed=29, drift_axis=0,
                                  drift_beta_per_slot=np.full(ppc, 0.99))
    sim = Simulation.from_plasma(pl, tuning=dict(tile=[4, 4, 1], halo=1, sort_every=1000))
    g, F, osp, _ = oracle_from_sim(sim)
    B.pic_stats(sim.ctx)
    terms = []
    for _ in range(8):
        sim.step(1)
        oracle.step(g, F, osp, terms=terms)
    strays = B.pic_stats(sim.ctx)
    assert strays > 0.3 * 8 * sum(s.n for s in osp)  # many updates strayed
    sim.check()
    Fg, spg = sim.download()
    compare_fields(Fg, F, floor=term_floor(g, terms))
    compare_particles(g, spg, osp)
    sim.close()


@pytest.mark.parametrize("tile,halo", [((8, 8, 4), 2), ((4, 4, 4), 1)])
def test_3d_strays_are_deferred_and_match_oracle(tile, halo):
    """3D tile kernels leave strays (stencil outside the tile window) to the
    deferred-particle kernel.  A hot plasma without re-sorting on a ragged box,
    with the fixed 8x8x4-tile window (halo 2) and the generic kernel (halo 1):
    particles and fields follow the oracle slot by slot, and strays occurred."""
    from paper_1906_06306_gb300 import binding as B
    from paper_1906_06306_gb300 import Simulation

    pl = workloads.uniform_plasma(3, 21, 19, 13, 0.45, 2, 0.01, 2.0, seed=27)
    sim = Simulation.from_plasma(pl, tuning=dict(tile=list(tile), halo=halo, sort_every=1000))
    g, F, osp, _ = oracle_from_sim(sim)
    B.pic_stats(sim.ctx)  # reset the counter
    terms = []
    for _ in range(5):
        sim.step(1)
        oracle.step(g, F, osp, terms=terms)
    assert B.pic_stats(sim.ctx) > 0
    sim.check()
    Fg, spg = sim.download()
    compare_fields(Fg, F, floor=term_floor(g, terms))
    compare_particles(g, spg, osp)
    sim.close()


def test_3d_split_path_defers_strays_and_matches_oracle():
    """pic_gather_push and pic_deposit in 3D after particles drifted out of
    their tile windows: the deferred kernel runs the strays in both modes (the
    push writes the pre-move snapshot, the deposit reads it)."""
    from paper_1906_06306_gb300 import binding as B
    from paper_1906_06306_gb300 import Simulation

    pl = workloads.uniform_plasma(3, 21, 19, 13, 0.45, 2, 0.01, 2.0, seed=28)
    sim = Simulation.from_plasma(pl, tuning=dict(tile=[8, 8, 4], halo=2, sort_every=1000))
    sim.step(4)
    g, F, osp, sp0 = oracle_from_sim(sim)
    B.pic_stats(sim.ctx)
    sim.gather_push()
    assert B.pic_stats(sim.ctx) > 0
    sim.deposit()
    sim.check()
    Fg, spg = sim.download()
    for o in osp:
        oracle.push_particles(g, F, o)
    compare_particles(g, spg, osp, xtol=2e-6, utol=2e-6)
    Fo = np.zeros_like(F)
    for s0, s1 in zip(sp0, spg):
        x_old = oracle.positions(g, s0["cell"], s0["off"])
        x_new = oracle.positions(g, s1["cell"], s1["off"])
        dx = periodic_dx(g, x_new, x_old)
        oracle.deposit(g, Fo, np.ascontiguousarray(x_old), np.ascontiguousarray(dx), s0["q"])
    for c in range(6, 9):
        assert rel_err(Fg[c] - F[c], Fo[c]) < 1e-5, c
    sim.close()


def test_edge_cases_tiny_grid_offsets_and_empty_species():
    """Grid smaller than a tile window (every particle takes the global path),
    offsets exactly 0 and just below 1, and an empty third species."""
    from paper_1906_06306_gb300 import Simulation

    rs = np.random.default_rng(26)
    nx, ny = 3, 2
    n = 40
    cell = rs.integers(0, nx * ny, size=n).astype(np.int32)
    off = rs.random((2, n)).astype(np.float32)
    off[:, :5] = 0.0
    off[:, 5:10] = workloads.plasma.ONE_MINUS
    u = rs.normal(scale=2.0, size=(3, n)).astype(np.float32)
    fields = np.zeros((9, 1, ny, nx), np.float32)
    fields[:6] = rs.normal(scale=0.1, size=(6, 1, ny, nx)).astype(np.float32)
    sp = [dict(q=-0.01, m=0.01, cell=cell, off=off, u=u),
          dict(q=0.01, m=0.01, cell=cell.copy(), off=off.copy(), u=-u),
          dict(q=0.01, m=0.01, cell=np.zeros(0, np.int32), off=np.zeros((2, 0), np.float32),
               u=np.zeros((3, 0), np.float32))]
    sim = Simulation(2, nx, ny, 1, 0.45, fields, sp, tuning=dict(sort_every=1000))
    g, F, osp, _ = oracle_from_sim(sim)
    terms = []
    for _ in range(5):
        sim.step(1)
        oracle.step(g, F, osp, terms=terms)
    Fg, spg = sim.download()
    compare_fields(Fg, F, floor=term_floor(g, terms))
    compare_particles(g, spg[:2], osp[:2])
    assert spg[2]["cell"].shape == (0,)
    sim.check()
    sim.close()


def test_invalid_particle_data_is_reported_not_used():
    from paper_1906_06306_gb300 import PicError, Simulation

    pl = workloads.uniform_plasma(2, 16, 16, 1, 0.45, 2, 0.01, 0.1, seed=27)
    pl.species[0].u[0, 3] = np.nan
    pl.species[1].off[0, 7] = 1.5
    sim = Simulation.from_plasma(pl)
    sim.step(1)
    with pytest.raises(PicError) as ei:
        sim.check()
    assert ei.value.status == 5
    assert "offset" in str(ei.value) and "four-velocity" in str(ei.value)
    sim.check()  # the status word was cleared
    sim.close()


def test_a_timed_out_device_wait_is_reported_and_the_context_stays_usable():
    """A bounded wait that runs out (one warp on a barrier that nothing
    completes) sets the timeout bit: pic_check reports PIC_ERR_TIMEOUT once,
    and the context then steps as a twin that never timed out (the same
    fields, energies and particles; slots inside a tile may be ordered
    differently by the two contexts' sorts)."""
    from paper_1906_06306_gb300 import PicError, Simulation, binding

    pl = workloads.turbulence_2d(n=48, ppc=4, r_p=4.0, theta=0.3, sigma=10.0, modes=4, seed=29)
    sim = Simulation.from_plasma(pl, tuning=dict(tile=[16, 8, 1]))
    twin = Simulation.from_plasma(pl, tuning=dict(tile=[16, 8, 1]))
    sim.step(1)
    twin.step(1)
    sim.check()
    binding.pic_wait_probe(sim.ctx)
    with pytest.raises(PicError) as ei:
        sim.check()
    assert ei.value.status == 4 and "wait" in str(ei.value)
    sim.check()  # the status word was cleared
    sim.step(3)
    twin.step(3)
    sim.check()
    Fa, spa = sim.download()
    Fb, spb = twin.download()
    np.testing.assert_allclose(Fa, Fb, rtol=0, atol=1e-5 * np.abs(Fb).max())
    np.testing.assert_allclose(sim.energies()[:4], twin.energies()[:4], rtol=1e-5)
    for a, b in zip(spa, spb):
        assert a["cell"].shape == b["cell"].shape
        assert (np.sort(a["cell"]) != np.sort(b["cell"])).sum() <= 4
        np.testing.assert_allclose(np.sort(a["u"], axis=1), np.sort(b["u"], axis=1), rtol=0,
                                   atol=1e-5 * np.abs(b["u"]).max())
    sim.close()
    twin.close()


def test_gauss_residual_stays_at_fp32_round_off():
    """Appendix B: with the charge-conserving deposit div E - rho keeps its
    initial value (0 for co-located pairs and E = 0).  In FP32 the residual is
    a random walk of round-off, far below the charge-separation signal."""
    from paper_1906_06306_gb300 import Simulation

    pl = workloads.turbulence_2d(n=64, ppc=8, r_p=4.0, theta=0.3, sigma=10.0, modes=4, seed=28)
    sim = Simulation.from_plasma(pl, tuning=dict(sort_every=10))
    sim.step(50)
    en = sim.energies()
    ns = sim.nspecies
    gauss_max = en[2 + ns]
    Fg, _ = sim.download()
    g = oracle.Grid(2, 64, 64, 1, 0.45)
    div_scale = np.abs(oracle.div_e(g, Fg.astype(np.float64))).max()
    assert div_scale > 1e-4
    assert gauss_max < 1e-4 * div_scale, (gauss_max, div_scale)
    sim.close()


def test_filtered_gauss_residual_3d():
    from paper_1906_06306_gb300 import Simulation

    pl = workloads.shock_3d(nx=24, ny=16, nz=16, ppc=2, seed=29)
    pl.species[0].u *= 0.1  # slow the flow so charge separates visibly
    sim = Simulation.from_plasma(pl, tuning=dict(tile=[8, 8, 8], filter_passes=2))
    sim.step(20)
    en = sim.energies()
    Fg, _ = sim.download()
    g = oracle.Grid(3, 24, 16, 16, 0.45)
    div_scale = np.abs(oracle.div_e(g, Fg.astype(np.float64))).max()
    assert en[2 + sim.nspecies] < 1e-4 * div_scale
    sim.close()


def test_full_size_turbulence_step_sampled_against_oracle():
    """The 1024^2, 16 particles per cell per species turbulence box in the
    benchmark's launch configuration: one fused pic_step; a sample of particles
    checked against the oracle's gather + Boris + move from the same state, and
    the full J lattice against the oracle's ZigZag of every GPU move."""
    from paper_1906_06306_gb300 import Simulation

    pl = workloads.turbulence_2d()
    sim = Simulation.from_plasma(pl)
    g, F, osp, sp0 = oracle_from_sim(sim)
    sim.step(1)
    sim.check()
    Fg, spg = sim.download()
    Fb = F.copy()
    oracle.push_half_b(g, Fb)
    rs = np.random.default_rng(30)
    for s0, s1, o in zip(sp0, spg, osp):
        pick = rs.choice(o.n, size=20000, replace=False)
        sub = oracle.Species(o.q, o.m, o.x[:, pick], o.u[:, pick])
        x_old, _ = oracle.push_particles(g, Fb, sub)
        u1 = s1["u"][:, pick].astype(np.float64)
        assert (np.abs(u1 - sub.u) <= 1e-5 * np.maximum(1.0, np.abs(sub.u))).all()
        x1 = oracle.positions(g, s1["cell"][pick], s1["off"][:, pick])
        assert np.abs(periodic_dx(g, x1, sub.x)).max() < 2e-5
    Jo = np.zeros_like(F)
    for s0, s1 in zip(sp0, spg):
        x_old = oracle.positions(g, s0["cell"], s0["off"])
        dx = np.zeros_like(x_old)
        dx[:2] = periodic_dx(g, oracle.positions(g, s1["cell"], s1["off"]), x_old)
        u = s1["u"].astype(np.float64)
        dx[2] = 0.45 * u[2] / np.sqrt(1.0 + (u * u).sum(0))
        oracle.deposit(g, Jo, x_old, dx, s0["q"])
    for c in range(6, 9):
        assert rel_err(Fg[c], Jo[c]) < 1e-5, c
    # Gauss residual after one step: FP32 rounding of E and of the current
    # terms, far below the field scale
    en = sim.energies()
    assert en[2 + sim.nspecies] < 1e-5 * max(np.abs(Fg[0:3]).max(), np.abs(Fg[6:9]).max())
    sim.close()


def test_shock_set_up_with_fdtd4_and_higuera_cary_matches_oracle():
    """The solver choice of the paper's shock run (Sect. 4.2): FDTD4 fields,
    Higuera-Cary pusher and Binomial2 filtering, on the cold Gamma = 10 flow."""
    from paper_1906_06306_gb300 import Simulation

    pl = workloads.shock_3d(nx=24, ny=12, nz=10, ppc=2, seed=32)
    sim = Simulation.from_plasma(pl, tuning=dict(tile=[8, 8, 4], sort_every=1000, filter_passes=2))
    sim.set_field_solver(4)
    sim.set_pusher("higuera_cary")
    g, F, osp, _ = oracle_from_sim(sim)
    oracle.set_field_order(4)
    oracle.set_pusher("higuera_cary")
    terms = []
    try:
        for k in range(1, 7):
            sim.step(1)
            oracle.step(g, F, osp, passes=2, terms=terms)
            Fg, spg = sim.download()
            compare_fields(Fg, F, floor=term_floor(g, terms))
            compare_particles(g, spg, osp)
    finally:
        oracle.set_field_order(2)
        oracle.set_pusher("boris")
    sim.check()
    sim.close()
