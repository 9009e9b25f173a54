"""pic_autotune picks launch parameters by timing real steps; the steps it
takes must advance the simulation exactly as pic_step does."""
import numpy as np
import pytest

import workloads

from gpu_helpers import compare_fields, current_scale, oracle_from_sim

pytestmark = pytest.mark.gpu

CANDIDATES = [dict(tile=[16, 16, 1], halo=3, sort_every=3),
              dict(tile=[8, 8, 1], halo=2, sort_every=5),
              dict(tile=[16, 8, 1], halo=2, sort_every=4)]


def _steps_taken(cands, steps):
    # two passes; per candidate 2 sort cycles untimed, then the timed whole cycles
    total = 0
    for c in cands:
        k = c["sort_every"]
        total += 2 * k + -(-max(steps, 2 * k) // k) * k
    return 2 * total


def test_autotune_advances_the_simulation_like_pic_step():
    from paper_1906_06306_gb300 import Simulation

    pl = workloads.turbulence_2d(n=48, ppc=4, r_p=4.0, theta=0.3, sigma=10.0, modes=4, seed=40)
    a = Simulation.from_plasma(pl)
    b = Simulation.from_plasma(pl)
    g, _, osp, _ = oracle_from_sim(a)
    chosen = a.autotune(CANDIDATES, steps=6)
    assert any(chosen["tile"][:2] == c["tile"][:2] and chosen["halo"] == c["halo"] and
               chosen["sort_every"] == c["sort_every"] for c in CANDIDATES)
    nsteps = _steps_taken(CANDIDATES, 6)
    b.step(nsteps)
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
