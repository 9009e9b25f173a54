"""Shock boundaries on the GPU (Sect. 4.2): conducting wall (reflection in
k_particles_deferred, field images) and receding injector (k_inject, the unsorted
tail kernel) against the FP64 oracle, plus the argument and state errors."""
import numpy as np
import pytest

import oracle
import workloads

from gpu_helpers import (compare_fields, compare_particles, current_scale, oracle_from_sim,
                         step_floor, term_floor)

pytestmark = pytest.mark.gpu


def _tube(dim, **kw):
    args = dict(dim=dim, nx=48, ny=8, nz=6, ppc=3, gamma_flow=3.0, theta=0.05, r_p=3.0,
                wall=3, x_inj=20, x_max=40.0, lt=8, filter_passes=0, seed=90 + dim)
    args.update(kw)
    return workloads.shock_tube(**args)


def _sim(pl, steps, **tuning):
    from paper_1906_06306_gb300 import Simulation

    cap = [s.n + workloads.injected_count(pl, steps + 2) for s in pl.species]
    sim = Simulation.from_plasma(pl, capacity=cap,
                                 tuning=dict(filter_passes=pl.meta["filter_passes"], **tuning))
    sim.set_shock_from_plasma(pl)
    return sim


@pytest.fixture
def oracle_wall():
    yield oracle.set_wall
    oracle.set_wall(0, 0)


@pytest.mark.parametrize("dim,passes", [(1, 0), (2, 0), (2, 2), (3, 1)])
def test_shock_tube_matches_oracle(oracle_wall, dim, passes):
    """Same particle slots on both sides (no sort during the run: the injected
    particles stay in the unsorted tail, appended in the same order), so
    particles, counts and fields compare one to one after 10 steps in which
    particles reflect at the wall and the injector lets new ones in."""
    pl = _tube(dim, filter_passes=passes)
    nsteps = 10
    sim = _sim(pl, nsteps, sort_every=1000)
    g, F, osp, _ = oracle_from_sim(sim)
    w, i_zero, inj = oracle.shock_from_plasma(pl)
    oracle_wall(w, i_zero)
    n0 = sim.counts()
    sim.step(nsteps)
    terms = []
    oracle.step_shock(g, F, osp, inj, 0, passes=passes, nsteps=nsteps, terms=terms)
    sim.check()
    counts = sim.counts()
    assert counts == [s.n for s in osp]
    assert counts[0] > n0[0]  # the injector let particles in
    Fg, spg = sim.download()
    compare_fields(Fg, F, floor=term_floor(g, terms))
    compare_particles(g, spg, osp)
    for s, o in zip(spg, osp):  # cell bookkeeping is exact (the oracle's cell of the GPU state)
        xg = oracle.positions(g, s["cell"], s["off"])
        assert xg[0].min() >= w
        assert np.array_equal(np.floor(xg[: g.dim]), np.floor(o.x[: g.dim])) or \
            np.mean(np.floor(xg[: g.dim]) != np.floor(o.x[: g.dim])) < 1e-3
    # reflections happened: particles that started in the wall's first cell
    # with u_x < 0 now move away from it
    reflected = sum(int(((s["u"][0] > 0) & (oracle.positions(g, s["cell"], s["off"])[0] < w + 5)).sum())
                    for s in spg)
    assert reflected > 0
    en, ref = sim.energies(), oracle.energies(g, F, osp)
    for a, b in zip(en[:2 + len(osp)], ref):
        assert abs(a - b) <= 1e-5 * max(abs(b), 1e-6 * sum(ref))
    sim.close()


def test_reflection_and_injection_alone_match_the_oracle(oracle_wall):
    """Zero fields, a handful of particles heading into the wall and a
    template entering: one step, J and every particle against the oracle."""
    from paper_1906_06306_gb300 import Simulation

    pl = _tube(2, ppc=1, x_inj=12, x_max=40.0, theta=1e-6, gamma_flow=5.0)
    rs = np.random.default_rng(3)
    for s in pl.species:  # put the fill right at the wall
        i = s.cell % pl.nx
        s.cell = (s.cell - i + pl.meta["shock"]["wall"]).astype(np.int32)
        s.off[0] = rs.uniform(0.0, 0.4, s.n).astype(np.float32)
    pl.species[1].off = pl.species[0].off.copy()
    sim = _sim(pl, 3, sort_every=1000)
    g, F, osp, _ = oracle_from_sim(sim)
    w, i_zero, inj = oracle.shock_from_plasma(pl)
    oracle_wall(w, i_zero)
    sim.step(1)
    terms = []
    oracle.step_shock(g, F, osp, inj, 0, nsteps=1, terms=terms)
    Fg, spg = sim.download()
    assert sim.counts() == [s.n for s in osp]
    compare_fields(Fg, F, floor=term_floor(g, terms))
    compare_particles(g, spg, osp)
    assert all((s["u"][0][: pl.species[0].n] > 0).all() for s in spg)  # every fill particle reflected
    sim.close()
    del Simulation


def test_sorted_run_matches_unsorted_run_and_oracle_statistics(oracle_wall):
    """With tile sorts every 3 steps (particles reordered, the tail folded into
    the tiles) the run equals the unsorted one up to summation order, and its
    counts equal the oracle's exactly."""
    pl = _tube(2, filter_passes=1)
    nsteps = 24
    a = _sim(pl, nsteps, sort_every=3)
    b = _sim(pl, nsteps, sort_every=1000)
    g, F, osp, _ = oracle_from_sim(b)
    w, i_zero, inj = oracle.shock_from_plasma(pl)
    oracle_wall(w, i_zero)
    a.step(nsteps)
    b.step(nsteps)
    terms = []
    oracle.step_shock(g, F, osp, inj, 0, passes=1, nsteps=nsteps, terms=terms)
    a.check()
    b.check()
    assert a.counts() == b.counts() == [s.n for s in osp]
    Fa, pa = a.download()
    Fb, pb = b.download()
    compare_fields(Fa, Fb.astype(np.float64), floor=step_floor(g, osp, nsteps))
    compare_fields(Fa, F, tol=1e-4, floor=term_floor(g, terms))
    for x, y in zip(pa, pb):
        ua = np.sort((x["u"].astype(np.float64) ** 2).sum(0))
        ub = np.sort((y["u"].astype(np.float64) ** 2).sum(0))
        assert np.abs(ua - ub).max() <= 1e-4 * max(1.0, ub.max())
        assert np.mean(np.sort(x["cell"]) != np.sort(y["cell"])) < 1e-2
    ea, eb = a.energies(), b.energies()
    for x, y in zip(ea[:4], eb[:4]):
        assert abs(x - y) <= 1e-4 * max(abs(y), 1e-6 * sum(eb[:4]))
    a.close()
    b.close()


@pytest.mark.parametrize("dim", [2, 3])
def test_gauss_law_on_the_plasma_side(dim):
    """pic_energies' Gauss residual covers wall < i < i_zero with the wall set;
    it stays at FP32 round-off of the charge-separation field."""
    pl = _tube(dim, filter_passes=2, nx=64, x_inj=30, x_max=58.0)
    sim = _sim(pl, 60, sort_every=4)
    sim.step(60)
    sim.check()
    en = sim.energies()
    ns = sim.nspecies
    F, _ = sim.download()
    w = pl.meta["shock"]["wall"]
    scale = max(np.abs(F[0:3, ..., w + 1:]).max(), np.abs(F[6:9]).max())
    assert scale > 0
    assert en[2 + ns] < 2e-5 * scale, (en[2 + ns], scale)
    sim.close()


def test_particles_behind_the_wall_are_flagged():
    from paper_1906_06306_gb300 import binding as B

    pl = _tube(2)
    s = pl.species[0]
    s.cell[0] = (s.cell[0] - s.cell[0] % pl.nx + 1)  # x cell 1 < wall = 3
    sim = _sim(pl, 2, sort_every=1000)
    sim.step(1)
    with pytest.raises(B.PicError) as ei:
        sim.check()
    assert ei.value.status == B.PIC_ERR_STATE
    sim.close()


def test_injection_beyond_the_capacity_is_refused():
    from paper_1906_06306_gb300 import Simulation
    from paper_1906_06306_gb300 import binding as B

    pl = _tube(2)
    sim = Simulation.from_plasma(pl, capacity=[s.n + 5 for s in pl.species])
    sim.set_shock_from_plasma(pl)
    with pytest.raises(B.PicError) as ei:
        sim.step(3)
    assert ei.value.status == B.PIC_ERR_ARG and "cap" in str(ei.value)
    sim.check()
    assert sim.counts() == [s.n for s in pl.species]
    sim.close()


def test_shock_contexts_refuse_batches_and_the_split_path():
    from paper_1906_06306_gb300 import Batch
    from paper_1906_06306_gb300 import binding as B

    pl = _tube(2)
    sim = _sim(pl, 2)
    with pytest.raises(B.PicError):
        Batch([sim])
    with pytest.raises(B.PicError) as ei:
        sim.gather_push()
    assert ei.value.status == B.PIC_ERR_STATE
    sim.close()


@pytest.mark.parametrize("bad,msg", [
    (dict(wall=0), "wall"),
    (dict(x_max=46.0), "x_max"),
    (dict(x0=2.0), "x0"),
    (dict(v_inj=8.0), "lt"),
    (dict(unsorted=True), "sorted"),
    (dict(bad_cell=True), "template cell"),
])
def test_set_shock_rejects_bad_arguments(bad, msg):
    from paper_1906_06306_gb300 import Simulation
    from paper_1906_06306_gb300 import binding as B

    pl = _tube(2)
    sh = pl.meta["shock"]
    sim = Simulation.from_plasma(pl)
    temps = [(t.cell.copy(), t.off.copy(), t.u.copy()) for t in sh["templates"]]
    if bad.get("unsorted"):
        temps[0][1][0, [0, -1]] = temps[0][1][0, [-1, 0]]
        temps[0][0][[0, -1]] = temps[0][0][[-1, 0]]
    if bad.get("bad_cell"):
        temps[1][0][0] = sh["lt"] * pl.ny * pl.nz
    args = dict(wall=sh["wall"], lt=sh["lt"], x0=sh["x_inj"], x_max=sh["x_max"],
                v_inj=sh["v_inj"], v_up=sh["v_up"])
    args.update({k: v for k, v in bad.items() if k in args})
    with pytest.raises(B.PicError) as ei:
        sim.set_shock(templates=temps, **args)
    assert ei.value.status == B.PIC_ERR_ARG and msg in str(ei.value)
    sim.close()


def test_full_size_shock_step_sampled_against_oracle(oracle_wall):
    """The 1024x128x128 shock set-up of the benchmark (wall on x = 1, injector
    from x = 512, 8 particles per cell per species, 4 filter passes, default
    3D launch configuration): one pic_step; sampled particles, including ones
    in the wall's cell that reflect, against the oracle's gather + Boris + move
    from the same state; every injected particle bit for bit against the
    oracle's injector; the Gauss residual on the plasma side."""
    from paper_1906_06306_gb300 import Simulation

    pl = workloads.shock_tube(dim=3, nx=1024, ny=128, nz=128, ppc=8, gamma_flow=10.0,
                              theta=1e-4, r_p=10.0, wall=1, x_inj=512, lt=64,
                              filter_passes=4, seed=1238)
    cap = [s.n + workloads.injected_count(pl, 3) for s in pl.species]
    sim = Simulation.from_plasma(pl, capacity=cap, tuning=dict(filter_passes=4))
    sim.set_shock_from_plasma(pl)
    F0, sp0 = sim.download()
    n0 = [s["cell"].shape[0] for s in sp0]
    sim.step(1)
    sim.check()
    F1, sp1 = sim.download()
    g = oracle.Grid(3, pl.nx, pl.ny, pl.nz, pl.c)
    w, i_zero, inj = oracle.shock_from_plasma(pl)
    oracle_wall(w, i_zero)
    Fb = F0.astype(np.float64)
    oracle.push_half_b(g, Fb)
    oracle.wall_fields(g, Fb, w, i_zero)
    rs = np.random.default_rng(31)
    reflected = 0
    for s0, s1, n in zip(sp0, sp1, n0):
        at_wall = np.flatnonzero(s0["cell"] % pl.nx == w)
        pick = np.concatenate([rs.choice(n, size=20000, replace=False),
                               rs.choice(at_wall, size=5000, replace=False)])
        sub = oracle.Species(s0["q"], s0["m"], oracle.positions(g, s0["cell"][pick], s0["off"][:, pick]),
                             s0["u"][:, pick].astype(np.float64))
        oracle.push_particles(g, Fb, sub)
        u1 = s1["u"][:, pick].astype(np.float64)
        assert (np.abs(u1 - sub.u) <= 1e-5 * np.maximum(1.0, np.abs(sub.u))).all()
        x1 = oracle.positions(g, s1["cell"][pick], s1["off"][:, pick])
        assert np.abs(x1 - sub.x).max() < 2e-5
        reflected += int((sub.u[0] > 0).sum())
    assert reflected > 1000  # the wall's cell holds particles that bounced
    # injection of step 0, bit for bit (same double-precision decisions)
    osp = [oracle.Species(s["q"], s["m"], np.zeros((3, 0)), np.zeros((3, 0))) for s in sp0]
    counts = inj.inject(0, osp)
    for s1, n, k, o in zip(sp1, n0, counts, osp):
        assert s1["cell"].shape[0] == n + k and k > 100000
        xg = oracle.positions(g, s1["cell"][n:], s1["off"][:, n:])
        assert np.array_equal(xg, o.x)
        assert np.array_equal(s1["u"][:, n:].astype(np.float64), o.u)
    # the pairs' currents cancel almost exactly, so FP32 rounding scales with
    # the per-species current c sum |q| n / ncells, not with the net field
    en = sim.energies()
    jscale = current_scale(g, [oracle.Species(s["q"], s["m"], np.zeros((3, n + k)), np.zeros((3, 1)))
                               for s, n, k in zip(sp1, n0, counts)])
    assert en[2 + sim.nspecies] < 1e-5 * jscale
    sim.close()


@pytest.mark.parametrize("dim", [2, 3])
def test_shock_tube_with_fdtd4_and_higuera_cary_matches_oracle(oracle_wall, dim):
    """The solver combination of the paper's shock run (FDTD4, Higuera-Cary,
    Binomial2) with the wall and the injector: FDTD4's wider stencil reads the
    conductor's mirror images two cells deep (wall at x = 3)."""
    pl = _tube(dim, filter_passes=2)
    nsteps = 8
    sim = _sim(pl, nsteps, sort_every=1000)
    sim.set_field_solver(4)
    sim.set_pusher("higuera_cary")
    g, F, osp, _ = oracle_from_sim(sim)
    w, i_zero, inj = oracle.shock_from_plasma(pl)
    oracle_wall(w, i_zero)
    oracle.set_field_order(4)
    oracle.set_pusher("higuera_cary")
    terms = []
    try:
        sim.step(nsteps)
        oracle.step_shock(g, F, osp, inj, 0, passes=2, nsteps=nsteps, terms=terms)
    finally:
        oracle.set_field_order(2)
        oracle.set_pusher("boris")
    sim.check()
    assert sim.counts() == [s.n for s in osp]
    Fg, spg = sim.download()
    compare_fields(Fg, F, floor=term_floor(g, terms))
    compare_particles(g, spg, osp)
    sim.close()
