"""The GPU discrete adjoint: one pic_adjoint_step against the oracle's
adjoint step; the checkpointed reverse sweep's gradient of the magnetic energy
against the oracle's gradient and central differences of the oracle's forward
run; the torch.autograd wrapper; and the cases the adjoint refuses."""
import numpy as np
import pytest

import oracle
import workloads

from gpu_helpers import oracle_from_sim, random_fields

pytestmark = pytest.mark.gpu

SHAPES = {1: (1, 1, 26), 2: (1, 12, 14), 3: (6, 7, 8)}


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)


def _random_sim(dim, seed, passes):
    from paper_1906_06306_gb300 import Simulation

    rs = np.random.default_rng(seed)
    nz, ny, nx = SHAPES[dim]
    pl = workloads.uniform_plasma(dim, nx, ny, nz, 0.45, 3, 0.02, 0.2, seed)
    pl.fields[:6] = random_fields((nz, ny, nx), rs)[:6]
    sim = Simulation.from_plasma(pl, tuning=dict(sort_every=1 << 30, filter_passes=passes))
    return sim, rs


@pytest.mark.parametrize("dim,passes", [(1, 0), (2, 0), (2, 2), (3, 0), (3, 1)])
def test_adjoint_step_matches_oracle(dim, passes):
    import torch

    from paper_1906_06306_gb300 import binding as B

    sim, rs = _random_sim(dim, 300 + 10 * dim + passes, passes)
    g, F, osp, _ = oracle_from_sim(sim)
    shape = F.shape[1:]
    A = rs.normal(size=(9,) + shape).astype(np.float32)
    A[6:9] = 0.0
    xb = [rs.normal(size=(dim, s.n)).astype(np.float32) for s in osp]
    ub = [rs.normal(size=(3, s.n)).astype(np.float32) for s in osp]
    At = torch.from_numpy(A).cuda()

    def rows(a, d):  # the library's layout: rows of the context's capacity
        t = torch.zeros((a.shape[0], d["cap"]), dtype=torch.float32)
        t[:, : a.shape[1]] = torch.from_numpy(a)
        return t.cuda()

    xbt = [rows(x, d) for x, d in zip(xb, sim.species)]
    ubt = [rows(u, d) for u, d in zip(ub, sim.species)]
    Fw = sim.fields.clone()
    asp = [B.pic_adjoint_species(d["cell"].data_ptr(), d["off"].data_ptr(), d["u"].data_ptr(),
                                 x.data_ptr(), u.data_ptr())
           for d, x, u in zip(sim.species, xbt, ubt)]
    B.pic_adjoint_step(sim.ctx, Fw.data_ptr(), asp, At.data_ptr())
    torch.cuda.synchronize()
    A64 = A.astype(np.float64)
    xb64 = [np.zeros((3, s.n)) for s in osp]
    for a, x in zip(xb64, xb):
        a[:dim] = x
    ub64 = [u.astype(np.float64) for u in ub]
    oracle.adj_step(g, F, osp, xb64, ub64, A64, passes=passes)
    Ag = At.cpu().numpy()
    assert np.abs(Ag[6:9]).max() == 0.0
    assert _rel(Ag[0:6], A64[0:6]) < 2e-5
    for xg, xo, ug, uo in zip(xbt, xb64, ubt, ub64):
        n = uo.shape[1]
        assert _rel(xg.cpu().numpy()[:, :n], xo[:dim]) < 2e-5
        assert _rel(ug.cpu().numpy()[:, :n], uo) < 2e-5
    sim.close()


def _problem(nsteps=12, k=5):
    from paper_1906_06306_gb300 import Simulation
    from paper_1906_06306_gb300.adjoint import MagneticEnergyProblem

    pl, mf, amps = workloads.adjoint_box(n=16, ppc=2, theta=0.1, sigma=1.0, modes=3, seed=5)
    sim = Simulation.from_plasma(pl)
    return MagneticEnergyProblem(sim, mf, nsteps=nsteps, checkpoint_every=k), mf, amps


def _oracle_run(g, F0, sp0, nsteps):
    F = F0.copy()
    sp = [oracle.Species(s.q, s.m, s.x.copy(), s.u.copy()) for s in sp0]
    oracle.step(g, F, sp, nsteps=nsteps)
    return 0.5 * float((F[3:6] ** 2).sum())


def test_magnetic_energy_gradient_matches_oracle_and_differences():
    """Gradient with respect to the 9 mode amplitudes and every initial
    four-velocity after 12 steps (checkpoints every 5 steps): against the
    oracle's adjoint from the same initial state, and the amplitudes against
    central differences of the oracle's forward run.  The loss is smooth only
    between cell-face crossings of some particle (linear shape functions), so
    the differences use a step (1e-6, double precision) that no crossing
    falls within; with 1e-4 a few crossings already shift them by 0.3 %."""
    import torch

    prob, mf, amps = _problem()
    sim = prob.sim
    a = torch.tensor(amps, device=sim.device)
    loss = prob.run(a, prob.u0())
    g_a, g_u = prob.gradient()
    F0 = prob.adj.ckpt[0][0].cpu().numpy().astype(np.float64)
    g = oracle.Grid(sim.dim, sim.nx, sim.ny, sim.nz, sim.c)
    sp0 = [oracle.Species(d["q"], d["m"], oracle.positions(g, c.cpu().numpy(), o.cpu().numpy()),
                          u.cpu().numpy().astype(np.float64))
           for d, (c, o, u) in zip(sim.species, prob.adj.ckpt[0][1])]
    assert loss == pytest.approx(_oracle_run(g, F0, sp0, 12), rel=1e-5)

    def loss_grad(Ff, spf):
        A = g.zeros()
        A[3:6] = Ff[3:6]
        return A, [np.zeros((3, s.n)) for s in spf], [np.zeros((3, s.n)) for s in spf]

    F = F0.copy()
    sp = [oracle.Species(s.q, s.m, s.x.copy(), s.u.copy()) for s in sp0]
    A, xbar, ubar = oracle.gradient(g, F, sp, 12, loss_grad)
    mf64 = mf.astype(np.float64)
    go_a = (mf64 * A[3:6][None]).reshape(mf.shape[0], -1).sum(1)
    go_u = np.concatenate(ubar, axis=1)
    assert _rel(g_a.cpu().numpy(), go_a) < 1e-3
    assert _rel(g_u.cpu().numpy(), go_u) < 1e-3
    h = 1e-6
    for m in (0, 4):
        Fp, Fm = F0.copy(), F0.copy()
        Fp[3:6] += h * mf64[m]
        Fm[3:6] -= h * mf64[m]
        fd = (_oracle_run(g, Fp, sp0, 12) - _oracle_run(g, Fm, sp0, 12)) / (2 * h)
        assert go_a[m] == pytest.approx(fd, rel=1e-6)
        assert float(g_a[m]) == pytest.approx(fd, rel=1e-3)
    sim.close()


def test_full_size_gradient_matches_central_differences_of_the_gpu_run():
    """The differentiable set-up at its benchmark size (256^2 box, 32 particles
    per cell per species, theta 0.1, sigma 1, 64 modes, 200 steps, checkpoints
    every 20): the derivative of the loss along the normalised amplitude
    gradient, from the adjoint, against central differences (h = 1e-3) of the
    GPU's own forward run, along the gradient (where the difference signal is
    largest) and along a random direction.  Millions of particles average the
    kinks of the linear shape functions into a loss that is smooth at this
    step."""
    import torch

    from paper_1906_06306_gb300 import Simulation
    from paper_1906_06306_gb300.adjoint import MagneticEnergyProblem

    pl, mf, amps = workloads.adjoint_box(n=256, ppc=32, theta=0.1, sigma=1.0, modes=8, seed=1239)
    assert mf.shape[0] == 64 and pl.nparticles == 2 * 32 * 256 * 256
    sim = Simulation.from_plasma(pl)
    prob = MagneticEnergyProblem(sim, mf, nsteps=200, checkpoint_every=20)
    a = torch.tensor(amps, device=sim.device)
    u0 = prob.u0()
    prob.run(a, u0)
    g_a, _ = prob.gradient()
    norm = float(g_a.norm())
    v = g_a / norm
    h = 1e-3
    fd = (prob.run(a + h * v, u0) - prob.run(a - h * v, u0)) / (2 * h)
    assert fd == pytest.approx(norm, rel=0.01), (fd, norm)  # measured 0.18 %
    # a seeded random unit direction (about 5 % of the gradient's norm)
    rs = np.random.default_rng(1239)
    r = torch.tensor(rs.normal(size=64).astype(np.float32), device=sim.device)
    r = r / r.norm()
    fd = (prob.run(a + h * r, u0) - prob.run(a - h * r, u0)) / (2 * h)
    assert fd == pytest.approx(float((g_a * r).sum()), rel=0.05, abs=0.01 * norm)
    sim.close()


def test_autograd_function_gives_the_adjoint_gradient():
    import torch

    from paper_1906_06306_gb300.adjoint import MagneticEnergy

    prob, _, amps = _problem(nsteps=8, k=3)
    a = torch.tensor(amps, device=prob.sim.device, requires_grad=True)
    u = prob.u0().requires_grad_()
    loss = MagneticEnergy.apply(a, u, prob)
    loss.backward()
    prob.run(a.detach(), u.detach())
    g_a, g_u = prob.gradient()
    # the forward run is repeated, and its FP32 current sums are order
    # dependent, so the two gradients agree to rounding, not bit for bit
    assert float((a.grad - g_a).norm() / g_a.norm()) < 1e-4
    assert float((u.grad - g_u).norm() / g_u.norm()) < 1e-4
    prob.sim.close()


@pytest.mark.parametrize("change", ["fdtd4", "higuera_cary"])
def test_adjoint_refuses_what_it_does_not_model(change):
    import torch

    from paper_1906_06306_gb300 import binding as B

    sim, _ = _random_sim(2, 7, 0)
    if change == "fdtd4":
        sim.set_field_solver(4)
    else:
        sim.set_pusher("higuera_cary")
    A = torch.zeros_like(sim.fields)
    xb = [torch.zeros((2, d["cap"]), device="cuda") for d in sim.species]
    ub = [torch.zeros((3, d["cap"]), device="cuda") for d in sim.species]
    asp = [B.pic_adjoint_species(d["cell"].data_ptr(), d["off"].data_ptr(), d["u"].data_ptr(),
                                 x.data_ptr(), u.data_ptr()) for d, x, u in zip(sim.species, xb, ub)]
    with pytest.raises(B.PicError) as ei:
        B.pic_adjoint_step(sim.ctx, sim.fields.data_ptr(), asp, A.data_ptr())
    assert ei.value.status == B.PIC_ERR_STATE
    sim.close()
