"""Per-kernel timing of the field kernels on a grid with fields only (no
particles), through the public API and the library's own CUDA-event timers.

    python -m paper_1906_06306_gb300.microbench filter --grid 1024,128,128 --iters 50
    python -m paper_1906_06306_gb300.microbench fields --grid 1024,1024,1 --iters 200

`filter` runs the Binomial2 pass of the three current planes (Sect. 2.3.1,
Table 2): algorithmic bytes 3 planes read + 3 written = 24 B per cell.
`fields` runs the FDTD2 half step of B (24 B read, 12 B written per cell) and
the E update (36 B read, 12 B written).  The device holds the nine field
planes and one 3-plane filter buffer: 48 B per cell, so a 1024 x 128 x 128
box needs 0.8 GB and its current planes (201 MB) exceed L2.  One JSON line:
mean microseconds per launch and algorithmic GB/s per kernel.
"""
import argparse
import json

import numpy as np


def _sim(dim, n, seed):
    from .sim import Simulation

    nx, ny, nz = n
    rs = np.random.default_rng(seed)
    F = (0.01 * rs.normal(size=(9, nz, ny, nx))).astype(np.float32)
    sp = [dict(q=-1.0, m=1.0, cell=np.zeros(0, np.int32), off=np.zeros((dim, 0), np.float32),
               u=np.zeros((3, 0), np.float32))]
    return Simulation(dim, nx, ny, nz, 0.45, F, sp)


def run(kind, grid, iters, warmup=3):
    from . import binding as B

    n = list(grid) + [1] * (3 - len(grid))
    dim = 3 if n[2] > 1 else (2 if n[1] > 1 else 1)
    cells = n[0] * n[1] * n[2]
    sim = _sim(dim, n, 7)
    try:
        def work():
            if kind == "filter":
                sim.filter_current(1)
            else:
                sim.field_update(B.PIC_FIELD_B_HALF)
                sim.field_update(B.PIC_FIELD_E)

        for _ in range(warmup):
            work()
        B.pic_kernel_times(sim.ctx)  # reset the counters
        B.pic_timing(sim.ctx, True)
        for _ in range(iters):
            work()
        kt = B.pic_kernel_times(sim.ctx)
        B.pic_timing(sim.ctx, False)
    finally:
        sim.close()
    per_cell = {"filter": 24, "b_half": 36, "e_update": 48}
    out = {"grid": n, "cells": cells, "iters": iters}
    for k, (ms, launches) in kt.items():
        if launches == 0 or k not in per_cell:
            continue
        us = 1e3 * ms / launches
        out[k] = {"us_per_launch": us, "launches": int(launches),
                  "alg_bytes": per_cell[k] * cells, "alg_gbs": per_cell[k] * cells / us / 1e3}
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("kind", choices=["filter", "fields"])
    ap.add_argument("--grid", default="1024,128,128", help="nx[,ny[,nz]]")
    ap.add_argument("--iters", type=int, default=50)
    a = ap.parse_args(argv)
    print(json.dumps(run(a.kind, [int(v) for v in a.grid.split(",")], a.iters)))


if __name__ == "__main__":
    main()
