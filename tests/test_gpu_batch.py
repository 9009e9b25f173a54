"""Ensembles of independent boxes stepped as one CUDA graph (pic_batch_step)
against stepping each box alone with pic_step, and against the oracle."""
import numpy as np
import pytest

import oracle
import workloads

from gpu_helpers import compare_fields, oracle_from_sim, step_floor, term_floor

pytestmark = pytest.mark.gpu

BOXES = [(1, 96, 8, 3.0, 0.01), (2, 24, 4, 2.0, 0.05), (1, 200, 16, 5.0, 0.001),
         (2, 40, 6, 1.5, 0.1), (2, 17, 4, 8.0, 0.02), (1, 130, 10, 2.5, 0.03)]
CADENCE = [5, 10, 5, 2, 10, 5]  # lcm 10


def _boxes():
    return [workloads.weibel_box(d, n, ppc, g, t, seed=500 + i)
            for i, (d, n, ppc, g, t) in enumerate(BOXES)]


def _sims(plasmas):
    from paper_1906_06306_gb300 import Simulation

    return [Simulation.from_plasma(pl, tuning=dict(sort_every=k))
            for pl, k in zip(plasmas, CADENCE)]


def _same_state(sa, sb, nsteps):
    Fa, pa = sa.download()
    Fb, pb = sb.download()
    g = oracle.Grid(sa.dim, sa.nx, sa.ny, sa.nz, sa.c)
    osp = [oracle.Species(s["q"], s["m"], np.zeros((3, s["cell"].shape[0])),
                          np.zeros((3, s["cell"].shape[0]))) for s in pa]
    compare_fields(Fa, Fb.astype(np.float64), floor=step_floor(g, osp, nsteps))
    for x, y in zip(pa, pb):  # same particles; the order inside a tile may differ
        ua = np.sort((x["u"].astype(np.float64) ** 2).sum(0))
        ub = np.sort((y["u"].astype(np.float64) ** 2).sum(0))
        assert np.abs(ua - ub).max() <= 1e-5 * max(1.0, ub.max())
        assert np.array_equal(np.sort(x["cell"]), np.sort(y["cell"])) or \
            np.mean(np.sort(x["cell"]) != np.sort(y["cell"])) < 1e-3


def test_batch_matches_each_box_stepped_alone():
    from paper_1906_06306_gb300 import Batch

    plasmas = _boxes()
    batched, alone = _sims(plasmas), _sims(plasmas)
    batch = Batch(batched)
    nsteps = 27  # two graph launches of 10 steps, then 7 plain steps
    batch.step(nsteps)
    for s in alone:
        s.step(nsteps)
    for a, b in zip(batched, alone):
        a.check()
        _same_state(a, b, nsteps)
    # a tuning change on one box forces a new capture; results stay the same
    batched[1].set_tuning(halo=2)
    alone[1].set_tuning(halo=2)
    batch.step(20)
    for s in alone:
        s.step(20)
    for a, b in zip(batched, alone):
        _same_state(a, b, nsteps + 20)
    # so does a change of pusher and field solver on every box
    batch.set_pusher("higuera_cary")
    batch.set_field_solver(4)
    for s in alone:
        s.set_pusher("higuera_cary")
        s.set_field_solver(4)
    batch.step(10)
    for s in alone:
        s.step(10)
    for a, b in zip(batched, alone):
        _same_state(a, b, nsteps + 30)
    batch.close()
    for s in batched + alone:
        s.close()


def test_batch_with_a_3d_box_defers_strays_inside_the_graph():
    """A 3D box (hot plasma, halo 1: its tile kernel defers strays to the
    deferred-particle kernel, which then runs inside the captured graph)
    batched with a 2D one, against each stepped alone."""
    from paper_1906_06306_gb300 import Batch, Simulation

    plasmas = [workloads.uniform_plasma(3, 13, 11, 9, 0.45, 2, 0.01, 2.0, seed=520),
               _boxes()[1]]
    tun = [dict(tile=[4, 4, 4], halo=1, sort_every=5), dict(sort_every=5)]

    def make():
        return [Simulation.from_plasma(pl, tuning=t) for pl, t in zip(plasmas, tun)]

    batched, alone = make(), make()
    batch = Batch(batched)
    batch.step(12)
    for s in alone:
        s.step(12)
    for a, b in zip(batched, alone):
        a.check()
        _same_state(a, b, 12)
    batch.close()
    for s in batched + alone:
        s.close()


def test_full_ensemble_batched_matches_sampled_boxes_alone():
    """The benchmark's ensemble (256 uneven 1D/2D Weibel boxes, 252.7 M
    particles) stepped as one batch, in the launch configuration of the
    benchmark (one graph per sort cycle of all boxes): a seeded sample of
    boxes against the same boxes stepped alone, over two sort cycles."""
    from paper_1906_06306_gb300 import Batch, Simulation

    recipe = workloads.weibel_ensemble(count=256)
    plasmas = [workloads.weibel_box(*b) for b in recipe]
    assert sum(p.nparticles for p in plasmas) > 2.5e8
    batched = [Simulation.from_plasma(p, tuning=dict(sort_every=10)) for p in plasmas]
    picks = sorted(np.random.default_rng(256).choice(256, size=6, replace=False))
    alone = [Simulation.from_plasma(plasmas[i], tuning=dict(sort_every=10)) for i in picks]
    batch = Batch(batched)
    batch.step(21)
    for s in alone:
        s.step(21)
    for i, s in zip(picks, alone):
        batched[i].check()
        _same_state(batched[i], s, 21)
    batch.close()
    for s in batched + alone:
        s.close()


def test_batched_box_follows_the_oracle():
    from paper_1906_06306_gb300 import Batch

    plasmas = _boxes()[:3]
    sims = _sims(plasmas)
    g, F, osp, _ = oracle_from_sim(sims[1])
    batch = Batch(sims)
    batch.step(10)
    terms = []
    oracle.step(g, F, osp, nsteps=10, terms=terms)
    Fg, _ = sims[1].download()
    compare_fields(Fg, F, floor=term_floor(g, terms))
    en = sims[1].energies()
    ref = oracle.energies(g, F, osp)
    for a, b in zip(en[:4], ref):
        assert abs(a - b) <= 1e-5 * max(abs(b), 1e-6 * sum(ref))
    batch.close()
    for s in sims:
        s.close()


def test_batch_rejects_mixed_streams_and_duplicates():
    import torch

    from paper_1906_06306_gb300 import binding as B
    from paper_1906_06306_gb300 import Simulation

    pl = _boxes()[0]
    a = Simulation.from_plasma(pl)
    other = torch.cuda.Stream()
    b = Simulation.from_plasma(pl, stream=other)
    with pytest.raises(B.PicError):
        B.pic_batch_create([a.ctx, a.ctx])
    h = B.pic_batch_create([a.ctx, b.ctx])
    with pytest.raises(B.PicError) as ei:
        B.pic_batch_step(h, 10, a.stream.cuda_stream)
    assert "stream" in str(ei.value)
    B.pic_batch_destroy(h)
    a.close()
    b.close()
