"""Gradients through many PIC steps by the discrete adjoint.

`Adjoint` runs a Simulation forward with a checkpoint of the state every K
steps; the reverse sweep recomputes each segment of K steps from its
checkpoint (keeping those K states) and runs pic_adjoint_step backwards over
them.  `MagneticEnergy` wraps it in a torch.autograd.Function: the magnetic
energy 0.5 sum B^2 after n steps as a function of the amplitudes of the
initial magnetic perturbation modes and of the initial four-velocities.

Every step, forward and adjoint, runs in libpic's kernels; PyTorch holds the
checkpoints and does the bookkeeping of the parametrisation (the initial
field as amplitudes times mode fields, and its transpose).
"""
from __future__ import annotations

import numpy as np

from . import binding as B

NO_SORT = 1 << 30  # sort cadence for adjoint runs: particle slots stay fixed


class Adjoint:
    """Forward run of `sim` with a checkpoint every `checkpoint_every` steps
    and the reverse sweep.  The steps themselves do not sort (the adjoint
    arrays follow the particle slots); with `tiled` (the default) the
    particles are tile-sorted in place every `sort_every` steps (a multiple of
    the checkpoint cadence, so that a sort opens a segment) by
    pic_sort_record, which keeps the permutation and the bucket starts: the
    forward steps and the adjoint's tile pass then run on tile-grouped
    particles, and the reverse sweep carries the gradients back through each
    sort's permutation (pic_adjoint_unsort).  Without it every adjoint step
    takes the global-memory pass.

    Memory is one state (fields and particles) per checkpoint plus the states
    of one segment; checkpoint_every=1 keeps every state of the forward run
    and recomputes nothing in the reverse sweep (for the 256^2 differentiable
    set-up about 0.1 GB a step)."""

    def __init__(self, sim, checkpoint_every: int = 20, tiled: bool = True,
                 sort_every: int | None = None):
        if checkpoint_every < 1:
            raise ValueError("checkpoint_every must be >= 1")
        if sort_every is None:  # the first multiple of the checkpoint cadence from 20 on
            sort_every = -(-20 // checkpoint_every) * checkpoint_every
        if tiled and (sort_every < 1 or sort_every % checkpoint_every):
            raise ValueError("sort_every must be a positive multiple of checkpoint_every")
        self.sim = sim
        self.K = int(checkpoint_every)
        self.S = int(sort_every)
        self.tiled = bool(tiled)
        self.nsteps = 0
        self.ckpt = []
        sim.set_tuning(sort_every=NO_SORT)

    def _sort(self):
        """Tile sort in place, recorded: (perm, tstart) per species (None for a
        species without particles)."""
        s = self.sim
        torch = s.torch
        nb = B.pic_sort_bins(s.ctx)
        perm, tst = [], []
        for n in s.counts():
            perm.append(torch.empty(n, dtype=torch.int32, device=s.device) if n else None)
            tst.append(torch.empty(nb + 1, dtype=torch.int32, device=s.device) if n else None)
        B.pic_sort_record(s.ctx, [p.data_ptr() if p is not None else 0 for p in perm],
                          [t.data_ptr() if t is not None else 0 for t in tst])
        return perm, tst

    def _assume(self, rec):
        if rec is not None:
            B.pic_sort_assume(self.sim.ctx, [t.data_ptr() if t is not None else 0 for t in rec[1]])

    def _state(self):
        s = self.sim
        return (s.fields.clone(),
                [(d["cell"].clone(), d["off"].clone(), d["u"].clone()) for d in s.species])

    def _restore(self, st):
        F, sp = st
        self.sim.fields.copy_(F)
        for d, (c, o, u) in zip(self.sim.species, sp):
            d["cell"].copy_(c)
            d["off"].copy_(o)
            d["u"].copy_(u)

    def forward(self, nsteps: int):
        """nsteps steps of the simulation, keeping a checkpoint every K (taken
        after the tile sort that opens it every S steps, which it records)."""
        self.nsteps = int(nsteps)
        self.ckpt = []
        for t in range(self.nsteps):
            if t % self.K == 0:
                rec = self._sort() if self.tiled and t % self.S == 0 else None
                self.ckpt.append((self._state(), rec))
            self.sim.step(1)

    def zeros(self):
        """Adjoint buffers for the current simulation: (fields [9, ...],
        xbar per species [D, cap], ubar per species [3, cap]), zero."""
        torch = self.sim.torch
        A = torch.zeros_like(self.sim.fields)
        xb = [torch.zeros((self.sim.dim, d["cap"]), dtype=torch.float32, device=self.sim.device)
              for d in self.sim.species]
        ub = [torch.zeros((3, d["cap"]), dtype=torch.float32, device=self.sim.device)
              for d in self.sim.species]
        return A, xb, ub

    def backward(self, A, xbar, ubar):
        """Reverse sweep: A, xbar, ubar hold the gradient with respect to the
        final state and are turned, in place, into the gradient with respect
        to the state at the start of the forward run.  The simulation is left
        at the final state."""
        sim = self.sim
        final = self._state()
        # the grouping each segment's particles are in: that of the last sort
        # at or before the segment
        groups, g = [], None
        for _, rec in self.ckpt:
            g = rec if rec is not None else g
            groups.append(g)
        for seg in reversed(range(len(self.ckpt))):
            t0 = seg * self.K
            t1 = min(self.nsteps, t0 + self.K)
            st, rec = self.ckpt[seg]
            states = [st]  # the checkpoint is the segment's first state
            if t1 - t0 > 1:  # recompute the others (not the step past the last)
                self._restore(st)
                self._assume(groups[seg])
                for k in range(t1 - t0 - 1):
                    sim.step(1)
                    states.append(self._state())
            tst = groups[seg][1] if groups[seg] is not None else [None] * len(xbar)
            for F, sp in reversed(states):
                asp = [B.pic_adjoint_species(c.data_ptr(), o.data_ptr(), u.data_ptr(),
                                             xb.data_ptr(), ub.data_ptr(),
                                             t.data_ptr() if t is not None else None)
                       for (c, o, u), xb, ub, t in zip(sp, xbar, ubar, tst)]
                B.pic_adjoint_step(sim.ctx, F.data_ptr(), asp, A.data_ptr())
            if rec is not None:  # back through the sort that opened the segment
                asp = [B.pic_adjoint_species(None, None, None, xb.data_ptr(), ub.data_ptr())
                       for xb, ub in zip(xbar, ubar)]
                B.pic_adjoint_unsort(sim.ctx, [p.data_ptr() if p is not None else 0
                                               for p in rec[0]], asp)
        self._restore(final)
        if groups:
            self._assume(groups[-1])
        return A, xbar, ubar


class MagneticEnergyProblem:
    """The differentiable set-up: a Simulation whose initial B is
    base B + sum_m amps[m] modes[m] and whose initial four-velocities are
    given, run for nsteps with checkpoints every K.  modes: float32 array
    [M, 3, nz, ny, nx] of B perturbation fields (planes Bx, By, Bz)."""

    def __init__(self, sim, modes, nsteps: int, checkpoint_every: int = 20,
                 sort_every: int | None = None):
        torch = sim.torch
        self.sim = sim
        self.adj = Adjoint(sim, checkpoint_every, sort_every=sort_every)
        self.nsteps = int(nsteps)
        self.modes = torch.as_tensor(np.asarray(modes, dtype=np.float32), device=sim.device)
        self.base_fields = sim.fields.clone()
        self.base = [(d["cell"].clone(), d["off"].clone()) for d in sim.species]
        self.counts = sim.counts()

    def u0(self):
        """Initial four-velocities of every species, concatenated: [3, N]."""
        return self.sim.torch.cat([d["u"][:, :n].clone() for d, n in zip(self.sim.species,
                                                                         self.counts)], dim=1)

    def run(self, amps, u0):
        """Set the initial state from (amps, u0), run forward, return the
        magnetic energy 0.5 sum B^2 (FP64 reduction on the GPU)."""
        sim = self.sim
        F = self.base_fields.clone()
        F[3:6] += (amps.to(F.dtype)[:, None, None, None, None] * self.modes).sum(0)
        sim.fields.copy_(F)
        off = 0
        for d, (c, o), n in zip(sim.species, self.base, self.counts):
            d["cell"].copy_(c)
            d["off"].copy_(o)
            d["u"][:, :n].copy_(u0[:, off:off + n].to(d["u"].dtype))
            off += n
        self.adj.forward(self.nsteps)
        return sim.energies()[1]

    def gradient(self, g=1.0):
        """Gradient of g * loss with respect to (amps, u0) after run()."""
        A, xb, ub = self.adj.zeros()
        A[3:6] = g * self.sim.fields[3:6]
        self.adj.backward(A, xb, ub)
        torch = self.sim.torch
        g_amps = (self.modes * A[3:6][None]).flatten(1).sum(1)
        g_u0 = torch.cat([u[:, :n] for u, n in zip(ub, self.counts)], dim=1)
        return g_amps, g_u0


def _make_function():
    import torch

    class MagneticEnergy(torch.autograd.Function):
        """loss = MagneticEnergy.apply(amps, u0, problem): the magnetic energy
        after problem.nsteps steps; backward by the discrete adjoint."""

        @staticmethod
        def forward(ctx, amps, u0, problem):
            ctx.problem = problem
            loss = problem.run(amps.detach(), u0.detach())
            return torch.tensor(loss, dtype=torch.float64, device=amps.device)

        @staticmethod
        def backward(ctx, grad):
            g_amps, g_u0 = ctx.problem.gradient(float(grad))
            return g_amps.to(torch.float32), g_u0.to(torch.float32), None

    return MagneticEnergy


def __getattr__(name):
    if name == "MagneticEnergy":
        fn = _make_function()
        globals()["MagneticEnergy"] = fn
        return fn
    raise AttributeError(name)
