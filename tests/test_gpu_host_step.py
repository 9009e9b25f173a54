"""pic_step_host, the end-to-end call from host memory (particles and fields
copied in, steps, copied back), against stepping the same state on the device
with pic_step; with rows longer than the particle count (cap) and with the
injector changing the counts between the copy in and the copy out."""
import numpy as np
import pytest

import workloads

from gpu_helpers import compare_fields, step_floor

pytestmark = pytest.mark.gpu


def _host_buffers(sim):
    """Pinned host copies of the device state, rows as long as the device's."""
    import torch

    from paper_1906_06306_gb300 import binding as B

    F, sp = sim.download()
    hs, keep = [], []
    for s, d in zip(sp, sim.species):
        arrs = []
        for k, rows in (("cell", 0), ("off", sim.dim), ("u", 3)):
            shape = (d["cap"],) if rows == 0 else (rows, d["cap"])
            a = torch.zeros(shape, dtype=torch.int32 if rows == 0 else torch.float32).pin_memory()
            a[..., : s[k].shape[-1]] = torch.from_numpy(s[k])
            arrs.append(a)
        keep.append(arrs)
        hs.append(B.pic_host_species(*[a.data_ptr() for a in arrs]))
    hf = torch.from_numpy(F).pin_memory()
    return hs, keep, hf


def _oracle_like(sim):
    import oracle

    return oracle.Grid(sim.dim, sim.nx, sim.ny, sim.nz, sim.c)


# (shock, dim, steps, sort cadence, particles per chunk, row padding): the
# periodic boxes take the overlapped copies, whose last step runs the particle
# kernel chunk by chunk (5000 particles per chunk: 4 chunks of the 2D box's
# 16,384 per species, 3 of the 3D box's; 2^22: one chunk); with a cadence of 2
# the last of 3 steps (and the only one of 1) opens a sort cycle; a padding
# makes the rows (cap) longer than the particle count
@pytest.mark.parametrize("shock,dim,nsteps,sort_every,chunk,pad",
                         [(False, 2, 4, 1000, 1 << 22, 0), (True, 2, 4, 1000, 1 << 22, 0),
                          (False, 3, 4, 1000, 1 << 22, 0), (False, 2, 3, 2, 1 << 22, 0),
                          (False, 2, 4, 1000, 5000, 0), (False, 2, 3, 2, 5000, 0),
                          (False, 2, 1, 2, 5000, 0), (False, 3, 3, 2, 5000, 0),
                          (False, 3, 4, 1000, 5000, 0), (False, 2, 3, 2, 5000, 77),
                          (False, 3, 2, 1000, 4096, 131)])
def test_step_host_equals_device_steps(shock, dim, nsteps, sort_every, chunk, pad):
    import oracle

    from paper_1906_06306_gb300 import Simulation
    from paper_1906_06306_gb300 import binding as B

    if shock:
        pl = workloads.shock_tube(dim=2, nx=48, ny=8, nz=1, ppc=3, gamma_flow=3.0, theta=0.05,
                                  r_p=3.0, wall=3, x_inj=20, x_max=40.0, lt=8, seed=93)
        cap = [s.n + workloads.injected_count(pl, 6) for s in pl.species]
    elif dim == 2:
        pl = workloads.turbulence_2d(n=64, ppc=4, r_p=4.0, theta=0.3, sigma=10.0, modes=4, seed=94)
        cap = [s.n + pad for s in pl.species] if pad else None
    else:  # hot 3D plasma, halo 1: strays go through the deferred-particle kernel
        pl = workloads.uniform_plasma(3, 21, 19, 13, 0.45, 2, 0.01, 2.0, seed=95)
        cap = [s.n + pad for s in pl.species] if pad else None
    tun = (dict(sort_every=sort_every) if dim == 2 else
           dict(tile=[4, 4, 4], halo=1, sort_every=sort_every))
    sims = []
    for _ in range(2):
        sim = Simulation.from_plasma(pl, capacity=cap, tuning=tun)
        if shock:
            sim.set_shock_from_plasma(pl)
        sims.append(sim)
    dev, host = sims
    if nsteps == 1:  # the set-up sort was at step 0: two steps to reach step 2's sort
        for sim in sims:
            sim.step(2)
    hs, keep, hf = _host_buffers(host)
    B.pic_set_host_chunk(host.ctx, chunk)
    B.pic_step_host(host.ctx, hs, hf.data_ptr(), nsteps)
    dev.step(nsteps)
    Fd, spd = dev.download()
    counts = dev.counts()
    assert host.counts() == counts
    g = _oracle_like(dev)
    osp = [oracle.Species(s["q"], s["m"], np.zeros((3, n)), np.zeros((3, 1))) for s, n in zip(spd, counts)]
    compare_fields(hf.numpy(), Fd.astype(np.float64), floor=step_floor(g, osp, nsteps))
    # the two contexts' initial tile sorts order particles differently inside a
    # tile, so the particles compare as multisets
    for s, arrs, n in zip(spd, keep, counts):
        cell, off, u = (a.numpy() for a in arrs)
        assert np.mean(np.sort(cell[:n]) != np.sort(s["cell"])) < 1e-3
        ua = np.sort((u[:, :n].astype(np.float64) ** 2).sum(0))
        ub = np.sort((s["u"].astype(np.float64) ** 2).sum(0))
        assert np.abs(ua - ub).max() <= 1e-5 * max(1.0, ub.max())
    for s in sims:
        s.close()
