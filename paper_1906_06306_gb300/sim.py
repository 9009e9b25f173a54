"""Device-resident PIC state driven through the C ABI.

PyTorch supplies device memory and the stream; every step of the path runs in
libpic's kernels.  A Simulation owns CUDA tensors for the 9 field planes and
each species' SoA arrays, created from host arrays (e.g. a workloads.Plasma).
"""
from __future__ import annotations

import numpy as np

from . import binding as B


class Simulation:
    """Periodic PIC box on one GPU.

    fields: float32[9, nz, ny, nx] (Ex Ey Ez Bx By Bz Jx Jy Jz);
    species: list of dicts with q, m, cell int32[n], off float32[D, n],
    u float32[3, n]."""

    def __init__(self, dim, nx, ny, nz, c, fields, species, device="cuda:0", stream=None,
                 tuning=None):
        import torch

        self.torch = torch
        self.dim, self.nx, self.ny, self.nz, self.c = dim, nx, ny, nz, float(c)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.fields = torch.from_numpy(np.ascontiguousarray(fields, dtype=np.float32)).to(self.device)
        self.species = []
        sps = []
        for s in species:
            d = dict(q=float(s["q"]), m=float(s["m"]),
                     cell=torch.from_numpy(np.ascontiguousarray(s["cell"], dtype=np.int32)).to(self.device),
                     off=torch.from_numpy(np.ascontiguousarray(s["off"], dtype=np.float32)).to(self.device),
                     u=torch.from_numpy(np.ascontiguousarray(s["u"], dtype=np.float32)).to(self.device))
            d["n"] = int(d["cell"].shape[0])
            self.species.append(d)
            sps.append(B.pic_species(d["q"], d["m"], d["n"], d["cell"].data_ptr(),
                                     d["off"].data_ptr(), d["u"].data_ptr()))
        grid = B.pic_grid(dim, nx, ny, nz)
        torch.cuda.synchronize(self.device)
        self.ctx = B.pic_init(grid, sps, self.c, 1.0, self.fields.data_ptr(), self.stream.cuda_stream)
        if tuning:
            self.set_tuning(**tuning)

    @classmethod
    def from_plasma(cls, pl, **kw):
        sp = [dict(q=s.q, m=s.m, cell=s.cell, off=s.off, u=s.u) for s in pl.species]
        return cls(pl.dim, pl.nx, pl.ny, pl.nz, pl.c, pl.fields, sp, **kw)

    @property
    def nspecies(self):
        return len(self.species)

    @property
    def nparticles(self):
        return sum(s["n"] for s in self.species)

    def set_tuning(self, tile=None, halo=0, sort_every=0, filter_passes=0, chunk=0):
        t = B.pic_tuning()
        if tile is not None:
            for d, v in enumerate(tile):
                t.tile[d] = int(v)
        t.halo, t.sort_every, t.filter_passes, t.chunk = halo, sort_every, filter_passes, chunk
        B.pic_set_tuning(self.ctx, t)

    def tuning(self):
        t = B.pic_get_tuning(self.ctx)
        return dict(tile=list(t.tile), halo=t.halo, sort_every=t.sort_every,
                    filter_passes=t.filter_passes, chunk=t.chunk)

    def autotune(self, candidates=None, steps=20):
        """Pick tile size, halo and sort cadence by timing real steps (they advance
        the simulation); returns the chosen tuning."""
        cs = None
        if candidates:
            cs = []
            for c in candidates:
                t = B.pic_tuning()
                for d, v in enumerate(c.get("tile", [0, 0, 0])):
                    t.tile[d] = int(v)
                t.halo, t.sort_every = c.get("halo", 0), c.get("sort_every", 0)
                t.chunk = c.get("chunk", 0)
                cs.append(t)
        B.pic_autotune(self.ctx, cs, steps)
        return self.tuning()

    def set_field_solver(self, order):
        """2 (FDTD2, default) or 4 (FDTD4)."""
        B.pic_set_field_solver(self.ctx, order)

    def set_pusher(self, name):
        """'boris' (default) or 'higuera_cary'."""
        B.pic_set_pusher(self.ctx, {"boris": B.PIC_PUSHER_BORIS,
                                    "higuera_cary": B.PIC_PUSHER_HIGUERA_CARY}[name])

    def step(self, n=1):
        B.pic_step(self.ctx, n)

    def sort(self):
        B.pic_sort(self.ctx)

    def gather_push(self):
        B.pic_gather_push(self.ctx)

    def deposit(self):
        B.pic_deposit(self.ctx)

    def filter_current(self, passes):
        B.pic_filter_current(self.ctx, passes)

    def field_update(self, which):
        B.pic_field_update(self.ctx, which)

    def energies(self):
        return B.pic_energies(self.ctx, self.nspecies)

    def check(self):
        B.pic_check(self.ctx)

    def download(self):
        """Host copies: (fields, [dict(cell, off, u) per species])."""
        self.stream.synchronize()
        sp = [dict(q=s["q"], m=s["m"], cell=s["cell"].cpu().numpy(), off=s["off"].cpu().numpy(),
                   u=s["u"].cpu().numpy()) for s in self.species]
        return self.fields.cpu().numpy(), sp

    def close(self):
        if getattr(self, "ctx", None) is not None:
            B.pic_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Ensemble of independent Simulations stepped together: each sort cycle
    of all boxes is one CUDA graph launch (pic_batch_step).  All simulations
    must use the same device and stream."""

    def __init__(self, sims):
        self.sims = list(sims)
        self.handle = B.pic_batch_create([s.ctx for s in self.sims])

    def set_field_solver(self, order):
        """Set the field solver of every box (the next step recaptures)."""
        for s in self.sims:
            s.set_field_solver(order)

    def set_pusher(self, name):
        """Set the pusher of every box (the next step recaptures)."""
        for s in self.sims:
            s.set_pusher(name)

    def step(self, n=1):
        B.pic_batch_step(self.handle, n, self.sims[0].stream.cuda_stream)

    def close(self):
        if getattr(self, "handle", None) is not None:
            B.pic_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
