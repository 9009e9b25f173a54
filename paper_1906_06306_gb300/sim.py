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
    u float32[3, n].  capacity (one per species, or None): row length of the
    device arrays, the room an injector (set_shock) may fill.  With
    align_rows the row length is rounded up to a multiple of 4, so that every
    row starts 16-byte aligned and the 1D/2D particle kernel can stream the
    records with bulk copies (without, rows of another length take its plain
    loads)."""

    def __init__(self, dim, nx, ny, nz, c, fields, species, device="cuda:0", stream=None,
                 tuning=None, capacity=None, align_rows=True):
        import torch

        self.torch = torch
        self.dim, self.nx, self.ny, self.nz, self.c = dim, nx, ny, nz, float(c)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.fields = torch.from_numpy(np.ascontiguousarray(fields, dtype=np.float32)).to(self.device)
        self.species = []
        sps = []
        for i, s in enumerate(species):
            n = int(np.asarray(s["cell"]).shape[0])
            cap = max(n, int(capacity[i])) if capacity is not None else n
            if align_rows:
                cap = (cap + 3) // 4 * 4
            if cap == n:
                cell = np.ascontiguousarray(s["cell"], dtype=np.int32)
                off = np.ascontiguousarray(s["off"], dtype=np.float32).reshape(dim, n)
                u = np.ascontiguousarray(s["u"], dtype=np.float32)
            else:
                cell = np.zeros(cap, dtype=np.int32)
                off = np.zeros((dim, cap), dtype=np.float32)
                u = np.zeros((3, cap), dtype=np.float32)
                cell[:n] = s["cell"]
                off[:, :n] = s["off"]
                u[:, :n] = s["u"]
            d = dict(q=float(s["q"]), m=float(s["m"]), n=n, cap=cap,
                     cell=torch.from_numpy(cell).to(self.device),
                     off=torch.from_numpy(off).to(self.device),
                     u=torch.from_numpy(u).to(self.device))
            self.species.append(d)
            sps.append(B.pic_species(d["q"], d["m"], n, d["cell"].data_ptr(),
                                     d["off"].data_ptr(), d["u"].data_ptr(), cap))
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

    def counts(self):
        """Current particle count of each species (grows with injection)."""
        return B.pic_particle_counts(self.ctx, self.nspecies)

    @property
    def nparticles(self):
        return sum(self.counts())

    def set_shock(self, wall, lt, x0, x_max, v_inj, v_up, templates):
        """Conducting wall and receding injector along x (Sect. 4.2).
        templates: one (cell int32[nt], off float32[D, nt], u float32[3, nt])
        per species, cells of an lt x ny x nz block, sorted by x."""
        sh = B.pic_shock()
        sh.wall, sh.lt = int(wall), int(lt)
        sh.x0, sh.x_max, sh.v_inj, sh.v_up = float(x0), float(x_max), float(v_inj), float(v_up)
        keep = []
        for i, (cell, off, u) in enumerate(templates):
            arrs = [np.ascontiguousarray(cell, dtype=np.int32),
                    np.ascontiguousarray(off, dtype=np.float32),
                    np.ascontiguousarray(u, dtype=np.float32)]
            keep.append(arrs)
            sh.nt[i] = arrs[0].shape[0]
            sh.tmpl[i] = B.pic_host_species(*[a.ctypes.data for a in arrs])
        B.pic_set_shock(self.ctx, sh)

    def set_shock_from_plasma(self, pl):
        """The wall and injector of a workloads.shock_tube plasma."""
        sh = pl.meta["shock"]
        self.set_shock(sh["wall"], sh["lt"], sh["x_inj"], sh["x_max"], sh["v_inj"], sh["v_up"],
                       [(t.cell, t.off, t.u) for t in sh["templates"]])

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
        """Host copies: (fields, [dict(cell, off, u) per species]) of the current
        particles."""
        self.stream.synchronize()
        ns = self.counts()
        sp = [dict(q=s["q"], m=s["m"], cell=s["cell"][:n].cpu().numpy(),
                   off=s["off"][:, :n].cpu().numpy(), u=s["u"][:, :n].cpu().numpy())
              for s, n in zip(self.species, ns)]
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
