"""Benchmark of the GB300 PIC step on the 2D3V decaying-turbulence workload
(1024 x 1024 cells, 16 particles per cell per species, theta = 0.3,
sigma = 10, forcing modes 1..8; Sect. 4.3 of arXiv:1906.06306).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is one full pic_step (B half step, fused gather + Boris + move +
ZigZag deposit, B half step, filter passes, E update, and the tile sort every
`sort_every` steps), over every particle.  value = particle-steps/s of the
whole job; for N > 1 (torchrun) every rank steps an independent replica of
the box ("replicas only": the single-GPU path has no exchange step).
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (gather+push+deposit), FP32 vs FP64 oracle, % HBM roofline"


def _turb(n):
    import workloads
    return workloads.turbulence_2d(n=n, seed=1235)


def _weibel(n):
    import workloads
    return workloads.weibel_1d(nx=n, seed=1234)


def _shock(n):
    import workloads
    return workloads.shock_3d(nx=n, ny=n // 8, nz=n // 8, seed=1236)


def _shock_tube(n):
    import workloads
    return workloads.shock_tube(dim=3, nx=n, ny=n // 8, nz=n // 8, ppc=8, gamma_flow=10.0,
                                theta=1e-4, r_p=10.0, wall=1, x_inj=n // 2,
                                lt=max(8, min(64, n // 16)), filter_passes=4, seed=1238)


# The set-ups of Sects. 4.1-4.3 at their benchmark sizes; the turbulence box is
# the one the headline metric is quoted on, the others are reported on request.
WORKLOADS = {
    "turbulence_2d3v": dict(make=_turb, dim=2, grid=1024, sample_grid=128, filter_passes=0,
                            desc=dict(ppc_per_species=16, species=2, theta=0.3, sigma=10.0,
                                      r_p=4.0, modes=8)),
    "weibel_1d3v": dict(make=_weibel, dim=1, grid=512, sample_grid=512, filter_passes=0,
                        desc=dict(ppc_per_species=64, species=2, theta=0.01, gamma_b=3.0,
                                  r_p=10.0)),
    "shock_3d3v_periodic": dict(make=_shock, dim=3, grid=1024, sample_grid=64, filter_passes=4,
                                desc=dict(ppc_per_species=8, species=2, theta=1e-4,
                                          gamma_flow=10.0, r_p=10.0)),
    # the shock set-up with its boundaries: conducting wall on the node x = 1
    # (one guard cell for the mirror image), receding injector moving at c
    # from x = nx/2 (the box starts half full), upstream template of 64 cells
    "shock_3d3v": dict(make=_shock_tube, dim=3, grid=1024, sample_grid=64, filter_passes=4,
                       shock=True,
                       desc=dict(ppc_per_species=8, species=2, theta=1e-4, gamma_flow=10.0,
                                 r_p=10.0, wall=1, injector_start="nx/2",
                                 injector_speed="c")),
}


def full_grid(name, n=0):
    """Grid of a workload at its benchmark size (or at size n): n, n x n, or
    n x n/8 x n/8 cells, as its recipe builds it."""
    w = WORKLOADS[name]
    n = n or w["grid"]
    return [n, n, n][:1] if w["dim"] == 1 else [n, n] if w["dim"] == 2 else [n, n // 8, n // 8]


def workload_config(name, pl):
    w = WORKLOADS[name]
    grid = [pl.nx, pl.ny, pl.nz][: pl.dim]
    return dict(workload=name, grid=grid, **w["desc"], filter_passes=w["filter_passes"])
FALLBACK_HBM_GBS = 6800.0
# committed ncu summaries of the fused particle kernel, per workload
PROFILES = {"turbulence_2d3v": os.path.join(ROOT, "profiles", "push_turbulence_2d3v.md"),
            "shock_3d3v": os.path.join(ROOT, "profiles", "push_shock_3d3v.md")}


def kernel_source_hash() -> str:
    """Hash of the particle kernel's sources with comments and whitespace
    removed: it changes when the code changes, not when a comment does."""
    import re

    h = hashlib.sha256()
    for f in ("pic_particles.cu", "pic_dev.cuh", "pic_kernels.h"):
        with open(os.path.join(ROOT, "paper_1906_06306_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update("".join(src.split()).encode())
    return h.hexdigest()[:16]


def launches_per_step(sim, shock=False):
    """Kernels of a graph-replayed pic_step on `sim`'s tuning, per step and per
    sort cycle: per step the first B half step, the tile particle kernel, one
    fused launch per filter pass, the deferred-particle kernel in 3D or with
    the wall, and the second B half step with the E update (two launches; on a
    periodic FDTD2 lattice of at most 4096 points one launch that also takes
    the next step's first B half step, whose launch then opens only each
    cycle); per sort and species the count, the scan (three kernels past 4096
    bins) and the scatter."""
    from paper_1906_06306_gb300 import binding as B

    tun = sim.tuning()
    cells = sim.nx * sim.ny * sim.nz
    small = not shock and cells <= 4096
    step = (1 if small else 3) + 1 + tun["filter_passes"] + (1 if sim.dim == 3 or shock else 0)
    sort = (3 if B.pic_sort_bins(sim.ctx) <= 4096 else 5) * sim.nspecies + (1 if small else 0)
    return step, sort


def profiled_traffic(workload, full_size, nparticles):
    """DRAM bytes per launch of the fused particle kernel from the workload's
    committed ncu summary, if it was taken on the current kernel source: the
    bytes of a full-size launch when the summary gives them, else its bytes per
    particle (a capture of a smaller box) times the particles of a launch."""
    try:
        txt = open(PROFILES[workload]).read()
    except (KeyError, OSError):
        return None
    vals = {}
    for line in txt.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_hash") != kernel_source_hash():
        return None
    try:
        if "dram_bytes_per_full_launch" in vals:
            return float(vals["dram_bytes_per_full_launch"]) if full_size else None
        return float(vals["dram_bytes_per_particle"]) * nparticles
    except (KeyError, ValueError):
        return None


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def job_value(seconds, units, dist=None, device=None):
    """Whole-job throughput of replicas: every rank processed `units` in
    `seconds`; the job took as long as its slowest rank (max over ranks) and
    processed the units of all ranks (sum).  Returns (max seconds, units/s)."""
    if dist is None:
        return seconds, units / seconds
    import torch

    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item()) / float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def host_cores() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_worker(name, n, target_s, steps, barrier):
    """One host process of the all-core oracle baseline: the workload's set-up
    on an n-box, calibrated to about target_s seconds (or `steps` steps),
    started together with the others; returns (particle-steps, seconds)."""
    import oracle

    w = WORKLOADS[name]
    pl = w["make"](n)
    g, F, sp = oracle.from_plasma(pl)
    run = _oracle_runner(w, pl, g, F, sp)
    k = steps
    if k <= 0:
        t0 = time.perf_counter()
        run(1)
        k = max(1, int(target_s / max(time.perf_counter() - t0, 1e-6)))
    barrier.wait()
    t0 = time.perf_counter()
    done = run(k)
    return done, time.perf_counter() - t0


def oracle_all_cores(name, n, target_s=10.0, steps=0, cores=None):
    """The FP64 oracle as it stands on every host core: one process per core
    (spawned, so that no CUDA state is inherited), each stepping its own copy
    of the seeded sample box; the processes start together behind a barrier.
    Returns (particle-steps/s summed over the processes, processes)."""
    import multiprocessing as mp

    import oracle

    oracle.build()  # once, before the workers load it
    cores = cores or host_cores()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        barrier = man.Barrier(cores)
        with ctx.Pool(cores) as pool:
            res = pool.starmap(_oracle_worker, [(name, n, target_s, steps, barrier)] * cores)
    return sum(d / t for d, t in res), cores


def cpu_baseline(name="turbulence_2d3v", steps=0, sample_grid=None, target_s=10.0,
                 all_cores=True):
    """The FP64 oracle, as it stands, on a sample of the same workload: the
    same set-up on a smaller box (same plasma per cell); `steps` steps, or as
    many as fit in about target_s seconds, on one host thread and (all_cores)
    on every host core, one process per core."""
    import oracle

    oracle.build()
    w = WORKLOADS[name]
    n = sample_grid or w["sample_grid"]
    pl = w["make"](n)
    g, F, sp = oracle.from_plasma(pl)
    run = _oracle_runner(w, pl, g, F, sp)
    t0 = time.perf_counter()
    run(1)
    one = time.perf_counter() - t0
    k = steps if steps > 0 else max(1, int(target_s / max(one, 1e-6)))
    t0 = time.perf_counter()
    done = run(k)
    dt = time.perf_counter() - t0
    box = "x".join(str(v) for v in [pl.nx, pl.ny, pl.nz][: pl.dim])
    sample = (f"{name} on a {box} box ({pl.nparticles} particles at the start, same plasma per "
              f"cell), FP64")
    one = {"value": done / dt, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
           "sample": f"{sample}, {k} steps, 1 host thread"}
    out = dict(one, seconds=dt, steps=k, particles=pl.nparticles, single_core=one)
    if all_cores and host_cores() > 1:
        v, cores = oracle_all_cores(name, n, target_s=target_s)
        out.update(value=v, cores=cores,
                   sample=f"{sample}: one process per host core, each stepping its own copy of "
                          f"the box for about {target_s:.0f} s")
    return out


def parity_report(name, steps=10, sample_grid=None):
    """The FP32 GPU path against the FP64 oracle, quantity by quantity, on the
    workload's CPU-baseline sample box (same set-up and seed, no tile sort so
    that particle slots match), over `steps` steps:

    - independent trajectories (the oracle steps its own FP64 state): the
      largest normwise error of each field component (max |GPU - oracle| /
      max |oracle|; and against the larger of max |oracle| and the running sum
      over the steps of the current's term scale, the field a step's currents
      can build, which is what matters where opposite charges cancel the
      current and the field stays near zero), of J against the largest sum of
      |ZigZag term| on any current word (oracle.deposit_abs; the scale FP32
      sums at), of the
      positions (cells) and four-velocities (relative to max(1, |u|)); at the
      last step each energy term and the Gauss-law residual on both sides;
    - the cell decisions where the two runs differ (a particle that ends
      within rounding of a cell face lands on either side of it in FP32 and
      FP64; ZigZag's relay point, Appendix D, then routes its current along
      another path, a jump of the order of one particle's current);
    - periodic boxes: J of each step against the oracle's deposit of the GPU's
      own moves (the same cell decisions), relative to the term scale."""
    import numpy as np

    import oracle
    import workloads
    from paper_1906_06306_gb300 import Simulation

    w = WORKLOADS[name]
    n = sample_grid or w["sample_grid"]
    pl = w["make"](n)
    shock = bool(w.get("shock"))
    cap = [s.n + workloads.injected_count(pl, steps + 2) for s in pl.species] if shock else None
    sim = Simulation.from_plasma(pl, capacity=cap,
                                 tuning=dict(filter_passes=w["filter_passes"], sort_every=10 ** 6))
    if shock:
        sim.set_shock_from_plasma(pl)
    F32, sp0 = sim.download()
    g = oracle.Grid(pl.dim, pl.nx, pl.ny, pl.nz, pl.c)
    F = F32.astype(np.float64)
    osp = [oracle.Species(s["q"], s["m"], oracle.positions(g, s["cell"], s["off"]),
                          s["u"].astype(np.float64)) for s in sp0]
    inj = None
    if shock:
        wall, i_zero, inj = oracle.shock_from_plasma(pl)
        oracle.set_wall(wall, i_zero)
    names = ["Ex", "Ey", "Ez", "Bx", "By", "Bz", "Jx", "Jy", "Jz"]
    ferr = dict.fromkeys(names, 0.0)
    fscale = dict.fromkeys(names, 0.0)
    jsum = 0.0
    jterm = dict.fromkeys(names[6:], 0.0)
    jsame = dict.fromkeys(names[6:], 0.0) if not shock else None
    xerr = uerr = 0.0
    flips, flip_steps = 0, []
    ext = np.array([pl.nx, pl.ny, pl.nz][: pl.dim], dtype=np.float64)[:, None]
    xg_old = [oracle.positions(g, s["cell"], s["off"]) for s in sp0]
    try:
        for k in range(steps):
            terms = []
            sim.step(1)
            oracle.step_shock(g, F, osp, inj, k, passes=w["filter_passes"], nsteps=1,
                              terms=terms)
            Fg, spg = sim.download()
            scale = float(terms[-1].max())
            jsum += scale
            for c, nm in enumerate(names):
                d = np.abs(Fg[c].astype(np.float64) - F[c])
                ref = np.abs(F[c]).max()
                ferr[nm] = max(ferr[nm], float(d.max() / ref) if ref > 0 else float(d.max()))
                big = max(ref, jsum if c < 6 else scale)
                fscale[nm] = max(fscale[nm], float(d.max() / big) if big > 0 else float(d.max()))
                if c >= 6 and scale > 0:
                    jterm[nm] = max(jterm[nm], float(d.max() / scale))
            xg_new = [oracle.positions(g, s["cell"], s["off"]) for s in spg]
            nflip = 0
            for s, o, xn in zip(spg, osp, xg_new):
                if o.n == 0:
                    continue
                dx = xn[: pl.dim] - o.x[: pl.dim]
                dx -= np.round(dx / ext) * ext
                xerr = max(xerr, float(np.abs(dx).max()))
                du = np.abs(s["u"].astype(np.float64) - o.u) / np.maximum(1.0, np.abs(o.u))
                uerr = max(uerr, float(du.max()))
                nflip += int((np.floor(xn[: pl.dim]) != np.floor(o.x[: pl.dim])).any(axis=0).sum())
            if nflip > flips:
                flip_steps.append(k + 1)
            flips = max(flips, nflip)
            if jsame is not None:  # the oracle's ZigZag of the GPU's moves
                Jm = g.zeros()
                for s, xo, xn in zip(spg, xg_old, xg_new):
                    mv = np.zeros_like(xo)
                    mv[: pl.dim] = xn[: pl.dim] - xo[: pl.dim]
                    mv[: pl.dim] -= np.round(mv[: pl.dim] / ext) * ext
                    u = s["u"].astype(np.float64)
                    mv[pl.dim:] = pl.c * u[pl.dim:] / np.sqrt(1.0 + (u * u).sum(axis=0))
                    oracle.deposit(g, Jm, np.ascontiguousarray(xo), np.ascontiguousarray(mv), s["q"])
                oracle.filter_binomial(g, Jm, w["filter_passes"])
                for c, nm in zip(range(6, 9), names[6:]):
                    d = np.abs(Fg[c].astype(np.float64) - Jm[c])
                    jsame[nm] = max(jsame[nm], float(d.max() / scale) if scale > 0 else 0.0)
            xg_old = xg_new
        en = sim.energies()
        ref = oracle.energies(g, F, osp)
        res = oracle.gauss_residual(g, F, osp, passes=w["filter_passes"])
        if shock:  # the plasma side: the wall node carries the conductor's surface charge
            res = res[..., wall + 1:i_zero]
        rho1 = float(np.abs(oracle.charge_density(g, osp[:1])).max())
    finally:
        if shock:
            oracle.set_wall(0, 0)
        sim.close()
    ns = len(osp)
    terms_names = ["E", "B"] + [f"K_species{s}" for s in range(ns)]
    total = sum(abs(v) for v in ref)
    energy = {nm: abs(a - b) / abs(b) if abs(b) > 1e-6 * total else abs(a - b) / total
              for nm, a, b in zip(terms_names, en[: 2 + ns], ref)}
    box = "x".join(str(v) for v in [pl.nx, pl.ny, pl.nz][: pl.dim])
    out = {"sample": f"{name} on a {box} box ({pl.nparticles} particles at the start), same "
                     f"seed as the workload, {steps} steps from the same FP32 state, no tile sort",
           "tolerance": 1e-5,
           "fields_max_rel": ferr, "fields_vs_current_scale": fscale, "J_vs_term_scale": jterm,
           "x_max_abs_cells": xerr, "u_max_rel": uerr, "energy_rel": energy,
           "cell_decision_flips": {"particles_max": flips, "first_at_steps": flip_steps},
           "gauss_max": {"gpu_fp64_reduction": float(en[2 + ns]),
                         "oracle": float(np.abs(res).max()),
                         "one_species_charge_density_max": rho1},
           "note": "energy terms below 1e-6 of the total are compared relative to the total; "
                   "J_vs_term_scale divides by the largest sum of |ZigZag term| on a word; "
                   "fields_vs_current_scale divides E and B by the larger of their maximum "
                   "and the running sum of that term scale over the steps, J by the larger "
                   "of its maximum and the step's term scale"}
    if jsame is not None:
        out["J_same_moves_vs_term_scale"] = jsame
    return out


def _oracle_runner(w, pl, g, F, sp):
    """run(k): k oracle steps of the workload (with the wall and injector of a
    shock set-up); returns the particle-steps done."""
    import oracle

    state = {"s": 0}
    if not w.get("shock"):
        def run(k):
            oracle.step(g, F, sp, passes=w["filter_passes"], nsteps=k)
            return sum(x.n for x in sp) * k
        return run
    wall, i_zero, inj = oracle.shock_from_plasma(pl)

    def run(k):
        oracle.set_wall(wall, i_zero)
        done = 0
        try:
            for _ in range(k):
                done += sum(x.n for x in sp)
                oracle.step_shock(g, F, sp, inj, state["s"], passes=w["filter_passes"])
                state["s"] += 1
        finally:
            oracle.set_wall(0, 0)
        return done
    return run


def ensemble_cpu_baseline(boxes=256, sample=4, target_s=12.0):
    """The FP64 oracle stepping a seeded sample of the ensemble's boxes one
    after the other (the oracle has no batched form), as many steps as fit in
    about target_s seconds."""
    import numpy as np

    import oracle
    import workloads

    oracle.build()
    recipe = workloads.weibel_ensemble(count=boxes)
    pick = sorted(np.random.default_rng(boxes).choice(len(recipe), size=sample, replace=False))
    states = []
    for i in pick:
        pl = workloads.weibel_box(*recipe[i])
        g, F, sp = oracle.from_plasma(pl)
        states.append((pl, g, F, sp))
    npart = sum(pl.nparticles for pl, _, _, _ in states)

    def run(k):
        for _, g, F, sp in states:
            oracle.step(g, F, sp, passes=0, nsteps=k)
        return npart * k

    t0 = time.perf_counter()
    run(1)
    one = time.perf_counter() - t0
    k = max(1, int(target_s / max(one, 1e-6)))
    t0 = time.perf_counter()
    done = run(k)
    dt = time.perf_counter() - t0
    desc = ", ".join(f"{pl.dim}D {pl.nx}" + (f"x{pl.ny}" if pl.dim == 2 else "")
                     for pl, _, _, _ in states)
    return {"value": done / dt, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"{sample} of the {boxes} ensemble boxes ({desc}; {npart} particles), "
                      f"stepped one after the other, {k} steps, FP64, 1 host thread"}


def run_reference(args):
    """The oracle as it stands on the host cores, K timed steps after W warm-up
    steps; each step runs the workload's set-up on a box small enough that the
    whole run stays within about 90 seconds."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import math

    import oracle

    oracle.build()
    w = WORKLOADS[args.workload]
    cal = cpu_baseline(args.workload, steps=1, all_cores=False)
    per_particle_step = 1.0 / cal["value"]
    budget = 90.0 / max(1, args.steps + args.warmup)
    # shrink the sample box until K + W steps fit the budget
    n = w["sample_grid"]
    parts = cal["particles"]
    while n > 16 and parts * per_particle_step > budget:
        n //= 2
        parts = max(1, parts // 2 ** w["dim"])
    pl = w["make"](n)
    cores = host_cores()
    value, secs = oracle_all_cores_steps(args.workload, n, args.steps, args.warmup, cores)
    box = "x".join(str(v) for v in [pl.nx, pl.ny, pl.nz][: pl.dim])
    sample = (f"{args.workload} on a {box} box ({pl.nparticles} particles, same plasma per cell) "
              f"per step and process, FP64, one process per host core ({cores}), each stepping "
              f"its own copy of the box")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "particle-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(workload_config(args.workload, pl),
                           grid=full_grid(args.workload, args.grid), sample=sample),
            "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": cores,
                             "kind": "oracle", "sample": sample,
                             "single_core": {"value": cal["value"], "cores": 1,
                                             "unit": "particle-steps/s",
                                             "sample": cal["sample"]}},
            "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _oracle_steps_worker(name, n, steps, warmup, barrier):
    """One process of the reference arm: `warmup` untimed steps of the set-up
    on an n-box, then, started together with the others, `steps` timed steps;
    returns (particle-steps, seconds)."""
    import oracle

    w = WORKLOADS[name]
    pl = w["make"](n)
    g, F, sp = oracle.from_plasma(pl)
    run = _oracle_runner(w, pl, g, F, sp)
    run(warmup)
    barrier.wait()
    t0 = time.perf_counter()
    done = run(steps)
    return done, time.perf_counter() - t0


def oracle_all_cores_steps(name, n, steps, warmup, cores):
    """The oracle on every host core for a fixed number of steps: returns
    (particle-steps/s summed over the processes, the slowest process's seconds)."""
    import multiprocessing as mp

    import oracle

    oracle.build()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        barrier = man.Barrier(cores)
        with ctx.Pool(cores) as pool:
            res = pool.starmap(_oracle_steps_worker, [(name, n, steps, warmup, barrier)] * cores)
    return sum(d / t for d, t in res), max(t for _, t in res)


def push_bytes_per_launch(pl, nparticles=None) -> float:
    """Algorithmic DRAM bytes of one fused particle launch: every particle's SoA
    record (int32 cell, D float offsets, 3 float u) read once and written once,
    the six E and B planes read once and the three J planes written once."""
    rec = 4 + 4 * pl.dim + 12
    n = pl.nparticles if nparticles is None else nparticles
    return float(n * 2 * rec + pl.ncells * (6 + 3) * 4)


def step_bytes(pl, nparticles, filter_passes, sort_every) -> float:
    """Algorithmic DRAM bytes of one whole pic_step: the fused particle launch
    (push_bytes_per_launch), the two B half steps (E and B read, B written: 36 B
    per cell; the first also clears J: 12 B more), the E update (E, B, J read, E
    written: 48 B), 24 B per cell for each filter pass, and the tile sort
    amortised over its cadence (the cell keys read to count, every record read
    and written by the scatter)."""
    rec = 4 + 4 * pl.dim + 12
    fields = pl.ncells * (36 + 48 + 48 + 24 * filter_passes)
    sort = nparticles * (4 + 2 * rec) / sort_every
    return push_bytes_per_launch(pl, nparticles) + fields + sort


def sub_record(name, steps, warmup, local=0):
    """A bounded run of another set-up at its benchmark size, in the same
    process as the headline: particle-steps/s and ms per step of `steps`
    pic_step calls (one pic_step(steps) call, i.e. CUDA-graph replay of whole
    sort cycles, where the box has no shock boundaries), then per-kernel
    CUDA-event times of a timed pass of per-step calls (pic_timing on) for the
    particle kernel's roofline; FP32 errors against the oracle on the
    set-up's CPU-baseline sample box."""
    import torch

    import workloads
    from paper_1906_06306_gb300 import Simulation
    from paper_1906_06306_gb300 import binding as B

    w = WORKLOADS[name]
    t_gen = time.perf_counter()
    pl = w["make"](w["grid"])
    gen_s = time.perf_counter() - t_gen
    shock = bool(w.get("shock"))
    kt_steps = min(steps, 100)
    cap = None
    if shock:
        cap = [s.n + workloads.injected_count(pl, warmup + steps + kt_steps + 4) for s in pl.species]
    dev = torch.device(f"cuda:{local}")
    sim = Simulation.from_plasma(pl, device=f"cuda:{local}",
                                 tuning=dict(filter_passes=w["filter_passes"]), capacity=cap)
    if shock:
        sim.set_shock_from_plasma(pl)
    del pl
    sim.step(warmup)
    torch.cuda.synchronize(dev)
    sim.check()
    tun = sim.tuning()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    done = 0
    t0.record(sim.stream)
    if shock:  # the injection grows the count every step
        for _ in range(steps):
            done += sum(sim.counts())
            sim.step(1)
    else:
        done = sum(sim.counts()) * steps
        sim.step(steps)
    t1.record(sim.stream)
    torch.cuda.synchronize(dev)
    ms = t0.elapsed_time(t1)
    clocks = sampler.stop()
    # per-kernel times (events around every launch: per-step calls, no graph)
    B.pic_kernel_times(sim.ctx)
    B.pic_timing(sim.ctx, True)
    kdone = 0
    for _ in range(kt_steps):
        kdone += sum(sim.counts())
        sim.step(1)
    torch.cuda.synchronize(dev)
    kt = B.pic_kernel_times(sim.ctx)
    B.pic_timing(sim.ctx, False)
    sim.check()
    sim.close()
    peak, peak_kind = hbm_peak()
    push_ms, push_n = kt["push"]
    avg_push_s = push_ms * 1e-3 / max(push_n, 1)
    avg_n = kdone / max(kt_steps, 1)
    geo = _Geometry(w["dim"], full_grid(name))
    alg = push_bytes_per_launch(geo, avg_n)
    return {
        "workload": name, "config": dict(workload_config(name, geo), particles_mean=avg_n,
                                         sort_every=tun["sort_every"], tile=tun["tile"][: w["dim"]],
                                         halo=tun["halo"], autotuned=False),
        "steps": steps, "warmup": warmup, "value": done / (ms * 1e-3),
        "unit": "particle-steps/s", "ms_per_step": ms / steps,
        "step_graph": not shock,
        "roofline": {"bound": "hbm", "achieved": alg / avg_push_s / 1e9, "peak": peak,
                     "unit": "GB/s", "frac": alg / avg_push_s / 1e9 / peak,
                     "traffic": profiled_traffic(name, geo.nx == 1024, avg_n),
                     "kernel": f"k_particles<{w['dim']},{3 if shock else 0}>",
                     "peak_source": peak_kind, "avg_launch_us": avg_push_s * 1e6,
                     "alg_bytes_per_launch": alg, "timed_steps": kt_steps},
        "kernel_ms_per_step": {k: v[0] / kt_steps for k, v in kt.items() if v[1] > 0},
        "clocks": clocks, "setup_s": gen_s,
    }


class _Geometry:
    """Cells of a box, for the byte counts (a Plasma's dim, extents, ncells)."""

    def __init__(self, dim, grid):
        self.dim = dim
        g = list(grid) + [1] * (3 - len(grid))
        self.nx, self.ny, self.nz = g
        self.ncells = self.nx * self.ny * self.nz


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    import workloads
    from paper_1906_06306_gb300 import Simulation
    from paper_1906_06306_gb300 import binding as B

    # every rank steps its own replica of the box; --grid changes its size for profiling runs
    w = WORKLOADS[args.workload]
    pl = w["make"](args.grid or w["grid"])
    shock = bool(w.get("shock"))
    tuning = dict(filter_passes=w["filter_passes"])
    if args.sort_every:
        tuning["sort_every"] = args.sort_every
    if args.tile:
        tuning["tile"] = [int(v) for v in args.tile.split(",")] + [1] * (3 - len(args.tile.split(",")))
    if args.halo:
        tuning["halo"] = args.halo
    cap = None
    if shock:  # room for every particle the injector lets in during this run
        total = args.warmup + args.steps + args.e2e_steps + 4
        cap = [s.n + workloads.injected_count(pl, total) for s in pl.species]
    sim = Simulation.from_plasma(pl, device=f"cuda:{local}", tuning=tuning, capacity=cap)
    if shock:
        sim.set_shock_from_plasma(pl)
    dev = torch.device(f"cuda:{local}")
    autotuned = args.autotune and not shock  # its steps would advance the shock: defaults
    if autotuned:  # untimed: real steps under candidate tunings, keeps the fastest
        sim.autotune(None, steps=40)
    tun = sim.tuning()
    for _ in range(args.warmup):
        sim.step(1)
    if not shock:  # one call of two sort cycles: the step graph is captured and replayed
        sim.step(2 * tun["sort_every"])
    torch.cuda.synchronize(dev)
    sim.check()

    # ---- device-resident timed region ----
    # Periodic boxes: one pic_step(K) call, as a user steps a simulation (CUDA-
    # graph replay of whole sort cycles); the per-kernel times come from a
    # separate pass of single steps with the library's event timers.  Shock
    # boundaries: single steps (the injection is planned on the host each step).
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    B.pic_kernel_times(sim.ctx)  # reset counters
    B.pic_stats(sim.ctx)  # reset the stray count
    if shock:
        B.pic_timing(sim.ctx, True)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    done = 0  # particle-steps: the count at the start of each step (host state, no sync)
    t0.record(sim.stream)
    if shock:
        for _ in range(args.steps):
            done += sum(sim.counts())
            sim.step(1)
    else:
        done = args.steps * sum(sim.counts())
        sim.step(args.steps)
    t1.record(sim.stream)
    torch.cuda.synchronize(dev)
    ms = t0.elapsed_time(t1)
    clocks = sampler.stop()
    strays = B.pic_stats(sim.ctx)  # particle updates that left their tile window
    if shock:
        kt = B.pic_kernel_times(sim.ctx)
        kt_steps = args.steps
        B.pic_timing(sim.ctx, False)
    else:  # the per-kernel pass (untimed as a whole)
        kt_steps = min(args.steps, 400)
        B.pic_timing(sim.ctx, True)
        for _ in range(kt_steps):
            sim.step(1)
        torch.cuda.synchronize(dev)
        kt = B.pic_kernel_times(sim.ctx)
        B.pic_timing(sim.ctx, False)
    if dist is not None:
        dist.barrier()
    sim.check()
    s_max, value = job_value(ms * 1e-3, done, dist, dev)
    ms_max = s_max * 1e3
    avg_n = done / max(args.steps, 1)

    # ---- the turbulence set-up at its stated sort cadence (every 20 steps) ----
    stated = None
    if args.workload == "turbulence_2d3v" and tun["sort_every"] != 20 and world == 1:
        sim.set_tuning(sort_every=20)
        sim.step(40)  # two cycles: graph capture and warm-up
        k = 200
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        c0.record(sim.stream)
        sim.step(k)  # CUDA-graph replay of whole sort cycles
        c1.record(sim.stream)
        torch.cuda.synchronize(dev)
        sms = c0.elapsed_time(c1)
        stated = {"sort_every": 20, "steps": k, "value": sum(sim.counts()) * k / (sms * 1e-3),
                  "unit": "particle-steps/s", "ms_per_step": sms / k,
                  "note": "the same box and tiles, one pic_step(200) call (graph replay)"}
        sim.set_tuning(sort_every=tun["sort_every"])
        sim.check()

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if args.e2e_steps > 0:
        F0, sp0 = sim.download()
        hs, keep = [], []
        for s, d in zip(sp0, sim.species):  # host rows as long as the device rows (cap)
            arrs = []
            for k, rows in (("cell", 0), ("off", pl.dim), ("u", 3)):
                shape = (d["cap"],) if rows == 0 else (rows, d["cap"])
                a = torch.zeros(shape, dtype=torch.int32 if rows == 0 else torch.float32).pin_memory()
                a[..., : s[k].shape[-1]] = torch.from_numpy(s[k])
                arrs.append(a)
            keep.append(arrs)
            hs.append(B.pic_host_species(*[a.data_ptr() for a in arrs]))
        hf = torch.from_numpy(F0).pin_memory()
        rec = 4 + 4 * pl.dim + 12
        if args.host_chunk > 0:
            B.pic_set_host_chunk(sim.ctx, args.host_chunk)
        B.pic_step_host(sim.ctx, hs, hf.data_ptr(), 1)  # warm-up
        if dist is not None:
            dist.barrier()
        e_done, h2d, d2h = 0, 0, 0
        te = time.perf_counter()
        for _ in range(args.e2e_steps):
            n_in = sum(sim.counts())
            B.pic_step_host(sim.ctx, hs, hf.data_ptr(), 1)
            n_out = sum(sim.counts())
            e_done += n_in
            h2d += n_in * rec + hf.numel() * 4
            d2h += n_out * rec + hf.numel() * 4
        e_s, e_value = job_value(time.perf_counter() - te, e_done, dist, dev)
        e2e = {"value": e_value, "unit": "particle-steps/s",
               "h2d_bytes_per_step": int(h2d // args.e2e_steps),
               "d2h_bytes_per_step": int(d2h // args.e2e_steps),
               "steps": args.e2e_steps,
               "note": "pic_step_host: pinned host particles + fields copied in, one step, copied back"}

    if rank != 0:
        sim.close()
        if dist is not None:
            dist.destroy_process_group()
        return 0

    push_ms, push_n = kt["push"]
    avg_push_s = push_ms * 1e-3 / max(push_n, 1)
    peak, peak_kind = hbm_peak()
    alg = push_bytes_per_launch(pl, avg_n)
    achieved = alg / avg_push_s / 1e9
    traffic = profiled_traffic(args.workload, pl.nx == 1024, avg_n)
    step_alg = step_bytes(pl, avg_n, tun["filter_passes"], tun["sort_every"])
    nsorts = -(-args.steps // tun["sort_every"])  # at most one sort per cadence in the loop
    per_step, per_sort = launches_per_step(sim, shock)
    launches = args.steps * per_step + nsorts * per_sort
    if shock:  # per step: 3 wall-field passes, the injection, and the tail kernel on
        # every step that does not start with a sort
        launches += args.steps * 4 + (args.steps - nsorts)
    wl = workload_config(args.workload, pl)
    line = {
        "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": dict(wl, particles=pl.nparticles if not shock else
                       {"start": pl.nparticles, "end": sum(sim.counts()), "mean_timed": avg_n},
                       sort_every=tun["sort_every"],
                       sort_every_source=("autotuned among 5, 10, 20 (the turbulence set-up"
                                          " states a sort every 20 steps: see at_stated_cadence)"
                                          if autotuned and args.workload == "turbulence_2d3v"
                                          else "autotuned" if autotuned else
                                          "library default or --sort-every"),
                       tile=tun["tile"][: pl.dim], halo=tun["halo"], autotuned=bool(autotuned),
                       strays_per_particle_step=strays / max(done, 1),
                       parallelism="replicas" if world > 1 else "single-gpu",
                       l2=("inputs larger than L2 (particle SoA %.2f GB), no flush" if
                           pl.nparticles * (16 + 4 * pl.dim) > 2 * 129e6 else
                           "working set fits in L2 (particle SoA %.3f GB): launch-latency bound,"
                           " no flush") % (pl.nparticles * (16 + 4 * pl.dim) / 1e9)),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": f"k_particles<{pl.dim},{3 if shock else 0}> (gather+push+move+deposit"
                               + (", conducting-wall variant)" if shock else ")"),
                     "peak_source": peak_kind, "avg_launch_us": avg_push_s * 1e6,
                     "alg_bytes_per_launch": alg},
        "step_roofline": {"bound": "hbm", "achieved": step_alg / (ms_max * 1e-3 / args.steps) / 1e9,
                          "peak": peak, "unit": "GB/s",
                          "frac": step_alg / (ms_max * 1e-3 / args.steps) / 1e9 / peak,
                          "alg_bytes_per_step": step_alg,
                          "note": "whole pic_step: particle kernel, field updates, filter passes"
                                  " and the tile sort amortised over its cadence"},
        "kernel_ms": {k: {"ms": v[0], "launches": v[1]} for k, v in kt.items()},
        "kernel_ms_steps": kt_steps,
        "gpu_launches": launches,
        "clocks": clocks,
        "e2e": e2e,
    }
    if stated is not None:
        line["at_stated_cadence"] = stated
    if world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(args.workload)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample",
                                                   "single_core")}
        line["parity"] = parity_report(args.workload)
    sim.close()
    if world == 1 and args.sub_records and args.workload == "turbulence_2d3v":
        # the other set-ups of the paper at their benchmark sizes, bounded runs
        line["other_workloads"] = {}
        for nm, k, wu in (("weibel_1d3v", 1000, 20), ("shock_3d3v", 20, 5)):
            rec = sub_record(nm, k, wu, local)
            if not args.no_cpu_baseline:
                rec["parity"] = parity_report(nm)
                cb = cpu_baseline(nm, target_s=5.0)
                rec["cpu_baseline"] = {k2: cb[k2] for k2 in ("value", "unit", "cores", "kind",
                                                              "sample", "single_core")}
            line["other_workloads"][nm] = rec
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_batched(args):
    """Ensemble of independent Weibel boxes of uneven sizes (1D lengths 128..4096,
    2D sides 32..256, 16..128 particles per cell per species, gamma_b 1.5..10,
    theta 0.001..0.1) stepped with pic_batch_step (one CUDA graph launch per sort
    cycle of all boxes), compared with stepping the boxes one after the other
    with pic_step.  Replicas only for N > 1."""
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    import workloads
    from paper_1906_06306_gb300 import Batch, Simulation

    recipe = workloads.weibel_ensemble(count=args.boxes)
    plasmas = [workloads.weibel_box(*b) for b in recipe]
    npart = sum(p.nparticles for p in plasmas)
    sims = [Simulation.from_plasma(p, device=f"cuda:{local}") for p in plasmas]
    cands = [dict(sort_every=k, halo=h) for k in (5, 10, 20) for h in (2, 3)]
    if args.autotune:
        for sm in sims:
            sm.autotune(cands, steps=10)
    batch = Batch(sims)
    dev = torch.device(f"cuda:{local}")
    stream = sims[0].stream
    batch.step(args.warmup)
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    batch.step(args.steps)
    t1.record(stream)
    torch.cuda.synchronize(dev)
    ms = t0.elapsed_time(t1)
    clocks = sampler.stop()
    # the same steps box by box, one pic_step call per box
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for sm in sims:
        sm.step(args.steps)
    s1.record(stream)
    torch.cuda.synchronize(dev)
    ms_seq = s0.elapsed_time(s1)
    for sm in sims:
        sm.check()
    s_max, value = job_value(ms * 1e-3, npart * args.steps, dist, dev)
    ms = s_max * 1e3
    alg = sum(float(p.nparticles * 2 * (4 + 4 * p.dim + 12) + p.ncells * 48) for p in plasmas)
    achieved = alg * args.steps / (ms * 1e-3) / 1e9
    peak, peak_kind = hbm_peak()
    cadences = sorted({sm.tuning()["sort_every"] for sm in sims})
    launches = 0
    for sm in sims:
        per_step, per_sort = launches_per_step(sm)
        launches += args.steps * per_step + -(-args.steps // sm.tuning()["sort_every"]) * per_sort
    line = {
        "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": dict(workload="batched_weibel", boxes=len(sims), particles=npart,
                       boxes_2d=sum(1 for p in plasmas if p.dim == 2), autotuned=bool(args.autotune),
                       sort_cadences=cadences, l2="inputs larger than L2, no flush",
                       parallelism="replicas" if world > 1 else "single-gpu"),
        "sequential": {"value": npart * args.steps / (ms_seq * 1e-3), "unit": "particle-steps/s",
                       "ms_per_step": ms_seq / args.steps,
                       "note": "same boxes and steps, one pic_step(K) call per box in turn"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "whole step of all boxes (graph replay; per-kernel events are not"
                               " recorded inside graphs)", "peak_source": peak_kind},
        "gpu_launches": launches,
        "clocks": clocks, "e2e": None,
    }
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = ensemble_cpu_baseline(len(sims))
        print(json.dumps(line), flush=True)
    batch.close()
    for sm in sims:
        sm.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_adjoint(args):
    """Gradient of the magnetic energy after --steps steps (200 for the 256^2
    box of the differentiable set-up: 32 particles per cell per species,
    theta 0.1, sigma 1, 64 seeded modes of dB ~ 0.1 B0) with respect to the 64
    mode amplitudes and every initial four-velocity: forward run keeping every
    state where half the free device memory holds them, else a checkpoint
    every 20 steps (tile sorts every 20 steps, recorded), then the reverse
    sweep (recomputed segments, if any, and adjoint steps).  value =
    particle-steps of the forward run per second of forward + reverse.
    Replicas only for N > 1."""
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    import workloads
    from paper_1906_06306_gb300 import Simulation
    from paper_1906_06306_gb300 import binding as B
    from paper_1906_06306_gb300.adjoint import MagneticEnergy, MagneticEnergyProblem

    n = args.grid or 256
    pl, mf, amps = workloads.adjoint_box(n=n, ppc=32, theta=0.1, sigma=1.0, modes=8, seed=1239)
    dev = torch.device(f"cuda:{local}")
    sim = Simulation.from_plasma(pl, device=f"cuda:{local}")
    # every state of the forward run is kept when half the free device memory
    # holds them (about 0.1 GB a step on the 256^2 box: 20 GB for 200 steps),
    # so that the reverse sweep recomputes nothing; else a checkpoint every 20
    # steps; tile sorts every 20 steps
    state_bytes = pl.nparticles * 24 + pl.ncells * 36
    kcp = 1 if (args.steps + 1) * state_bytes <= 0.5 * torch.cuda.mem_get_info(dev)[0] else 20
    prob = MagneticEnergyProblem(sim, mf, nsteps=args.warmup, checkpoint_every=kcp, sort_every=20)
    a = torch.tensor(amps, device=dev)
    u0 = prob.u0()
    prob.run(a, u0)  # warm-up: a short gradient (--warmup steps), then a full-length one,
    prob.gradient()  # after which the allocator holds the kept states' memory
    prob.nsteps = args.steps
    prob.run(a, u0)
    prob.gradient()
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    B.pic_kernel_times(sim.ctx)
    B.pic_timing(sim.ctx, True)
    t0, t1, t2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    t0.record(sim.stream)
    loss = prob.run(a, u0)
    t1.record(sim.stream)
    g_a, g_u = prob.gradient()
    t2.record(sim.stream)
    torch.cuda.synchronize(dev)
    ms_f, ms_b = t0.elapsed_time(t1), t1.elapsed_time(t2)
    kt = B.pic_kernel_times(sim.ctx)
    B.pic_timing(sim.ctx, False)
    clocks = sampler.stop()
    npart = pl.nparticles
    s_max, value = job_value((ms_f + ms_b) * 1e-3, npart * args.steps, dist, dev)
    ms = s_max * 1e3
    # end to end through the autograd function: parameters from pinned host
    # memory, gradients back to the host
    ha = torch.from_numpy(amps).pin_memory()
    hu = u0.cpu().pin_memory()
    te = time.perf_counter()
    ad = ha.to(dev, non_blocking=True).requires_grad_()
    ud = hu.to(dev, non_blocking=True).requires_grad_()
    lo = MagneticEnergy.apply(ad, ud, prob)
    lo.backward()
    ga_h, gu_h = ad.grad.cpu(), ud.grad.cpu()
    e_s, e_value = job_value(time.perf_counter() - te, npart * args.steps, dist, dev)
    adj_ms, adj_n = kt["adjoint"]
    avg_adj = adj_ms * 1e-3 / max(adj_n, 1)
    # kernels behind the library's timed calls: a push is the tile kernel (2D,
    # periodic: no deferred-particle kernel), an adjoint step (tile pass) the B
    # rebuild, 2 adjoint B half steps, the adjoint E update, one per filter
    # pass, a bucket check per species, the tile pass and the deferred pass
    passes = sim.tuning()["filter_passes"]
    launches = (kt["push"][1] + kt["b_half"][1] + kt["e_update"][1] + kt["filter"][1] +
                kt["sort"][1] + (6 + passes + sim.nspecies) * kt["adjoint"][1])
    # per adjoint step: particle state read (4 + 8 + 12 B) and gradients read and
    # written (2 x (8 + 12) B); E, B read and their gradients added once per cell
    alg = npart * (24 + 40) + pl.ncells * 4 * (6 + 9 + 12)
    peak, peak_kind = hbm_peak()
    line = {
        "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": dict(workload="adjoint_2d3v", grid=[n, n], ppc_per_species=32, species=2,
                       theta=0.1, sigma=1.0, modes=int(mf.shape[0]), checkpoint_every=kcp,
                       sort_every=20,
                       states_kept_gb=round((-(-args.steps // kcp) + (kcp if kcp > 1 else 0)) *
                                            state_bytes / 1e9, 1),
                       particles=npart, loss=float(loss),
                       grad_norm_amps=float(g_a.norm()), grad_norm_u0=float(g_u.norm()),
                       forward_ms=ms_f, reverse_ms=ms_b,
                       l2=("each adjoint step reads its own stored forward state (%.2f GB) and"
                           " the gradients (%.2f GB): %.2f GB per step, larger than L2; no flush")
                       % (npart * 24 / 1e9, npart * 20 / 1e9, npart * 44 / 1e9),
                       parallelism="replicas" if world > 1 else "single-gpu"),
        "roofline": {"bound": "hbm", "achieved": alg / avg_adj / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": alg / avg_adj / 1e9 / peak, "traffic": None,
                     "kernel": "pic_adjoint_step (field adjoints + k_adj_particles)",
                     "peak_source": peak_kind, "avg_launch_us": avg_adj * 1e6,
                     "alg_bytes_per_launch": alg},
        "kernel_ms": {k: {"ms": v[0], "launches": v[1]} for k, v in kt.items()},
        "gpu_launches": launches,
        "clocks": clocks,
        "e2e": {"value": e_value, "unit": "particle-steps/s",
                "h2d_bytes_per_step": int((ha.numel() + hu.numel()) * 4 / args.steps),
                "d2h_bytes_per_step": int((ga_h.numel() + gu_h.numel()) * 4 / args.steps),
                "note": "MagneticEnergy.apply + backward from pinned host parameters"},
    }
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = adjoint_cpu_baseline()
        print(json.dumps(line), flush=True)
    sim.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def adjoint_cpu_baseline(n=32, nsteps=40):
    """The oracle's gradient (forward states kept, adjoint sweep) of the same
    loss on a small box of the same plasma (one host thread)."""
    import numpy as np

    import oracle
    import workloads

    oracle.build()
    pl, mf, amps = workloads.adjoint_box(n=n, ppc=32, theta=0.1, sigma=1.0, modes=8, seed=1239)
    g, F, sp = oracle.from_plasma(pl)
    F[3:6] += np.tensordot(amps.astype(np.float64), mf.astype(np.float64), axes=1)

    def loss_grad(Ff, spf):
        A = g.zeros()
        A[3:6] = Ff[3:6]
        return A, [np.zeros((3, s.n)) for s in spf], [np.zeros((3, s.n)) for s in spf]

    t0 = time.perf_counter()
    oracle.gradient(g, F, sp, nsteps, loss_grad)
    dt = time.perf_counter() - t0
    return {"value": pl.nparticles * nsteps / dt, "unit": "particle-steps/s", "cores": 1,
            "kind": "oracle",
            "sample": f"adjoint_2d3v gradient on a {n}x{n} box ({pl.nparticles} particles), "
                      f"{nsteps} steps forward + adjoint, FP64, 1 host thread"}


def micro_run(kind, grid, iters, warmup=3):
    """Per-kernel timing of the field kernels on a box with fields only (no
    particles), through the public API and the library's own CUDA-event
    timers.  `filter`: one Binomial2 pass of the three current planes
    (Table 2), 3 planes read + 3 written = 24 B per cell.  `fields`: the FDTD2
    half step of B (24 B read, 12 B written per cell) and the E update (36 B
    read, 12 B written).  The device holds the nine field planes and one
    3-plane filter buffer, 48 B per cell (a 1024 x 128 x 128 box: 0.8 GB, its
    current planes 201 MB, more than L2).  Returns the mean microseconds per
    launch and algorithmic GB/s of each kernel."""
    import numpy as np

    from paper_1906_06306_gb300 import Simulation
    from paper_1906_06306_gb300 import binding as B

    n = list(grid) + [1] * (3 - len(grid))
    dim = 3 if n[2] > 1 else (2 if n[1] > 1 else 1)
    cells = n[0] * n[1] * n[2]
    rs = np.random.default_rng(7)
    F = (0.01 * rs.normal(size=(9, n[2], n[1], n[0]))).astype(np.float32)
    sp = [dict(q=-1.0, m=1.0, cell=np.zeros(0, np.int32), off=np.zeros((dim, 0), np.float32),
               u=np.zeros((3, 0), np.float32))]
    sim = Simulation(dim, n[0], n[1], n[2], 0.45, F, sp)
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
    out = {"micro": kind, "grid": n, "cells": cells, "iters": iters}
    for k, (ms, launches) in kt.items():
        if launches == 0 or k not in per_cell:
            continue
        us = 1e3 * ms / launches
        out[k] = {"us_per_launch": us, "launches": int(launches),
                  "alg_bytes": per_cell[k] * cells, "alg_gbs": per_cell[k] * cells / us / 1e3}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--sort-every", type=int, default=0, help="0 = library default / autotuned")
    ap.add_argument("--tile", type=str, default="",
                    help="tile extents, e.g. 16,8 (with --no-autotune: fix the tuning that "
                         "autotuning picks, for profiling runs)")
    ap.add_argument("--halo", type=int, default=0, help="0 = library default / autotuned")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the default tuning instead of autotuning before the timed region")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--host-chunk", type=int, default=0,
                    help="particles per chunk of the end-to-end call's overlapped copies "
                         "(0 = library default)")
    ap.add_argument("--no-sub-records", dest="sub_records", action="store_false",
                    help="skip the bounded 1D Weibel and 3D shock runs of the default line")
    ap.add_argument("--grid", type=int, default=0,
                    help="box size (2D side, 1D length, 3D x-length with y = z = x/8); "
                         "0 = the workload's benchmark size")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["batched_weibel", "adjoint_2d3v"],
                    default="turbulence_2d3v")
    ap.add_argument("--boxes", type=int, default=256, help="boxes of the batched_weibel ensemble")
    ap.add_argument("--micro", choices=["filter", "fields"], default="",
                    help="time one kind of field kernel alone (no particles) and exit")
    ap.add_argument("--micro-grid", default="1024,128,128", help="nx[,ny[,nz]] for --micro")
    ap.add_argument("--micro-iters", type=int, default=50)
    args = ap.parse_args()
    if args.micro:
        print(json.dumps(micro_run(args.micro, [int(v) for v in args.micro_grid.split(",")],
                                   args.micro_iters)))
        return 0
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        if args.workload == "adjoint_2d3v":
            rank, _, _ = dist_env()
            if rank == 0:
                cb = adjoint_cpu_baseline()
                print(json.dumps({"impl": "reference", "metric": METRIC, "value": cb["value"],
                                  "unit": cb["unit"], "n_gpus": args.gpus, "steps": args.steps,
                                  "warmup": args.warmup, "higher_is_better": True,
                                  "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                                  "data": "synthetic",
                                  "config": {"workload": "adjoint_2d3v",
                                             "grid": [args.grid or 256, args.grid or 256],
                                             "ppc_per_species": 32, "species": 2, "theta": 0.1,
                                             "sigma": 1.0, "modes": 64, "checkpoint_every": 1,
                                             "sort_every": 20,
                                             "sample": cb["sample"]},
                                  "cpu_baseline": cb,
                                  "e2e": {"value": cb["value"], "unit": cb["unit"],
                                          "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
            return 0
        if args.workload == "batched_weibel":
            rank, _, _ = dist_env()
            if rank == 0:
                cb = ensemble_cpu_baseline(args.boxes)
                print(json.dumps({"impl": "reference", "metric": METRIC, "value": cb["value"],
                                  "unit": cb["unit"], "n_gpus": args.gpus, "steps": args.steps,
                                  "warmup": args.warmup, "higher_is_better": True,
                                  "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                                  "data": "synthetic",
                                  "config": {"workload": "batched_weibel", "boxes": args.boxes,
                                             "sample": cb["sample"]},
                                  "cpu_baseline": cb,
                                  "e2e": {"value": cb["value"], "unit": cb["unit"],
                                          "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
            return 0
        return run_reference(args)
    if args.workload == "batched_weibel":
        return run_batched(args)
    if args.workload == "adjoint_2d3v":
        return run_adjoint(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
