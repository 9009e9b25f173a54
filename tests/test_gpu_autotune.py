"""pic_autotune picks launch parameters by timing real steps; the steps it
takes must advance the simulation exactly as pic_step does."""
import numpy as np
import pytest

import workloads

from gpu_helpers import compare_fields, current_scale, oracle_from_sim

pytestmark = pytest.mark.gpu

# short cadences: the autotuner takes 4 cycles of each candidate (two passes
# of 2 untimed + 2 timed), 40 steps in all; over many more steps the two runs'
# float-atomic orders drift apart in the turbulent plasma beyond the tolerance
CANDIDATES = [dict(tile=[16, 16, 1], halo=3, sort_every=2),
              dict(tile=[8, 8, 1], halo=2, sort_every=1),
              dict(tile=[16, 8, 1], halo=2, sort_every=2)]


def _replay_autotune(sim, cands, steps, chosen):
    """The steps pic_autotune documents, taken through set_tuning and step: two
    passes over the candidates (the second in reverse order), each candidate
    re-tuned, stepped two sort cycles, then max(steps, 2 cycles) rounded up to
    whole cycles; at the end the chosen tuning is set."""
    orig = sim.tuning()
    for order in (cands, cands[::-1]):
        for c in order:
            k = c["sort_every"]
            sim.set_tuning(tile=c["tile"], halo=c["halo"], sort_every=k,
                           filter_passes=orig["filter_passes"], chunk=orig["chunk"])
            sim.step(2 * k)
            sim.step(-(-max(steps, 2 * k) // k) * k)
    sim.set_tuning(tile=chosen["tile"], halo=chosen["halo"], sort_every=chosen["sort_every"],
                   filter_passes=orig["filter_passes"], chunk=orig["chunk"])


def test_autotune_advances_the_simulation_like_pic_step():
    from paper_1906_06306_gb300 import Simulation

    pl = workloads.turbulence_2d(n=48, ppc=4, r_p=4.0, theta=0.3, sigma=10.0, modes=4, seed=40)
    a = Simulation.from_plasma(pl)
    b = Simulation.from_plasma(pl)
    g, _, osp, _ = oracle_from_sim(a)
    chosen = a.autotune(CANDIDATES, steps=2)
    assert any(chosen["tile"][:2] == c["tile"][:2] and chosen["halo"] == c["halo"] and
               chosen["sort_every"] == c["sort_every"] for c in CANDIDATES)
    _replay_autotune(b, CANDIDATES, 2, chosen)
    assert a.tuning() == b.tuning()
    nsteps = 2 * sum(4 * c["sort_every"] for c in CANDIDATES)
    a.check()
    b.check()
    Fa, _ = a.download()
    Fb, _ = b.download()
    j = current_scale(g, osp)
    compare_fields(Fa, Fb.astype(np.float64), tol=1e-5,
                   floor=[nsteps * j] * 3 + [4 * 0.45 * nsteps * j] * 3 + [j] * 3)
    ea, eb = a.energies(), b.energies()
    for x, y in zip(ea[:4], eb[:4]):
        assert abs(x - y) <= 1e-5 * max(abs(y), 1e-6 * sum(eb[:4]))
    a.close()
    b.close()


def test_autotune_builtin_candidates_keep_filter_passes():
    from paper_1906_06306_gb300 import Simulation

    pl = workloads.shock_3d(nx=32, ny=16, nz=16, ppc=2, seed=41)
    sim = Simulation.from_plasma(pl, tuning=dict(filter_passes=2))
    chosen = sim.autotune(None, steps=2)
    assert chosen["filter_passes"] == 2
    sim.check()
    sim.close()
