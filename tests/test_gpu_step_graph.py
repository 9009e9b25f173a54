"""pic_step(n) replays whole sort cycles from a captured CUDA graph (boxes
without shock boundaries).  The graph holds the kernels of the plain step loop
with the same arguments, so a run through it equals the same run stepped one
call at a time, up to the order of particles inside a tile (a captured cycle
always opens with its sort); and it follows the oracle."""
import numpy as np
import pytest

import oracle
import workloads

from gpu_helpers import compare_fields, oracle_from_sim, step_floor, term_floor

pytestmark = pytest.mark.gpu


def _pair(pl, **tun):
    from paper_1906_06306_gb300 import Simulation

    return (Simulation.from_plasma(pl, tuning=dict(tun)),
            Simulation.from_plasma(pl, tuning=dict(tun)))


def _same(a, b, nsteps):
    Fa, pa = a.download()
    Fb, pb = b.download()
    g = oracle.Grid(a.dim, a.nx, a.ny, a.nz, a.c)
    osp = [oracle.Species(s["q"], s["m"], np.zeros((3, s["cell"].shape[0])), np.zeros((3, 1)))
           for s in pa]
    compare_fields(Fa, Fb.astype(np.float64), floor=step_floor(g, osp, nsteps))
    for x, y in zip(pa, pb):  # same particles; the order inside a tile may differ
        ua = np.sort((x["u"].astype(np.float64) ** 2).sum(0))
        ub = np.sort((y["u"].astype(np.float64) ** 2).sum(0))
        assert np.abs(ua - ub).max() <= 1e-5 * max(1.0, ub.max())
        assert np.array_equal(np.sort(x["cell"]), np.sort(y["cell"])) or \
            np.mean(np.sort(x["cell"]) != np.sort(y["cell"])) < 1e-3


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_graph_replay_equals_single_steps(dim):
    if dim == 1:
        pl = workloads.weibel_1d(nx=96, ppc=8, seed=60)
        tun = dict(sort_every=4)
    elif dim == 2:
        pl = workloads.turbulence_2d(n=40, ppc=4, r_p=4.0, theta=0.3, sigma=10.0, modes=4, seed=61)
        tun = dict(tile=[8, 8, 1], sort_every=5, filter_passes=1)
    else:
        pl = workloads.uniform_plasma(3, 17, 13, 11, 0.45, 2, 0.01, 2.0, seed=62)
        tun = dict(tile=[8, 8, 4], halo=2, sort_every=3)
    a, b = _pair(pl, **tun)
    k = tun["sort_every"]
    n = 4 * k + 1
    for _ in range(n):
        a.step(1)
    b.step(n)  # four graph launches and one plain step
    a.check()
    b.check()
    _same(a, b, n)
    # a tuning change invalidates the graph: both continue alike
    for s in (a, b):
        s.set_tuning(sort_every=k + 1)
    for _ in range(2 * (k + 1)):
        a.step(1)
    b.step(2 * (k + 1))
    _same(a, b, n + 2 * (k + 1))
    a.close()
    b.close()


@pytest.mark.parametrize("dim", [1, 2])
def test_chained_small_lattice_loop_equals_single_steps(dim):
    """On a periodic FDTD2 lattice of at most 4096 points the field launch of a
    step also runs the next step's first B half step inside one pic_step call;
    with the event timers on, pic_step(n) takes the plain loop (no graph), so
    this is the chained loop against calls of one step (never chained)."""
    from paper_1906_06306_gb300 import binding as B

    if dim == 1:
        pl = workloads.weibel_1d(nx=128, ppc=8, seed=64)
        tun = dict(sort_every=3)
    else:
        pl = workloads.turbulence_2d(n=32, ppc=4, r_p=4.0, theta=0.3, sigma=10.0, modes=4, seed=65)
        tun = dict(tile=[8, 8, 1], sort_every=4, filter_passes=1)
    a, b = _pair(pl, **tun)
    B.pic_timing(b.ctx, 1)
    n = 11
    for _ in range(n):
        a.step(1)
    b.step(n)
    B.pic_timing(b.ctx, 0)
    a.check()
    b.check()
    _same(a, b, n)
    a.close()
    b.close()


def test_graph_replay_follows_the_oracle():
    """Many steps through the graph with sorts in between, against the oracle:
    the fields after the run (particle order differs after sorts, fields do
    not)."""
    from paper_1906_06306_gb300 import Simulation

    pl = workloads.turbulence_2d(n=36, ppc=4, r_p=4.0, theta=0.3, sigma=1.0, modes=4, seed=63)
    sim = Simulation.from_plasma(pl, tuning=dict(tile=[8, 8, 1], sort_every=4))
    g, F, osp, _ = oracle_from_sim(sim)
    sim.step(16)
    terms = []
    oracle.step(g, F, osp, nsteps=16, terms=terms)
    sim.check()
    Fg, _ = sim.download()
    compare_fields(Fg, F, floor=term_floor(g, terms))
    en, ref = sim.energies(), oracle.energies(g, F, osp)
    for a, b in zip(en[:4], ref):
        assert abs(a - b) <= 1e-5 * max(abs(b), 1e-6 * sum(ref))
    sim.close()
