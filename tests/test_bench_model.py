"""The algorithmic byte models behind bench.py's roofline objects, written out
by hand for the 2D turbulence box (1024^2 cells, 33,554,432 particles) and a
3D box: the particle record is read and written once per step (4 B cell,
4 B per offset, 12 B u), the field kernels move fixed bytes per cell, and the
tile sort is amortised over its cadence."""
import os
import sys
from types import SimpleNamespace

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    sys.path.insert(0, ROOT)
    import bench

    return bench


def test_push_bytes_2d_turbulence_box():
    b = _bench()
    pl = SimpleNamespace(dim=2, nparticles=33554432, ncells=1024 * 1024)
    # 48 B per particle (2 x (4 + 8 + 12)), 36 B per cell (E, B read, J written)
    assert b.push_bytes_per_launch(pl) == 33554432 * 48 + 1048576 * 36 == 1648361472


def test_step_bytes_adds_fields_filter_and_amortised_sort():
    b = _bench()
    pl = SimpleNamespace(dim=3, nparticles=1000, ncells=64)
    push = 1000 * 2 * (4 + 12 + 12) + 64 * 36
    fields = 64 * (36 + 48 + 48 + 24 * 4)  # two B half steps (one clears J), E, 4 passes
    sort = 1000 * (4 + 2 * 28) / 3
    assert abs(b.step_bytes(pl, 1000, 4, 3) - (push + fields + sort)) < 1e-6
    # the fused launch at a different mean particle count
    assert b.push_bytes_per_launch(pl, 500) == 500 * 56 + 64 * 36


def test_launch_counts_per_step_and_per_sort_cycle(monkeypatch):
    """The claimed launch counts: 4 per step (first B half step, particle
    kernel, second B half step, E update), one per filter pass, the deferred
    kernel in 3D or with the wall; on a periodic FDTD2 lattice of at most 4096
    points 2 per step (particle kernel, one field launch that takes the next
    step's first B half step) and the first B half step once per sort cycle;
    per sort and species count, scan (3 kernels past 4096 bins) and scatter."""
    b = _bench()
    from paper_1906_06306_gb300 import binding as B

    def sim(dim, n, species, passes, bins):
        monkeypatch.setattr(B, "pic_sort_bins", lambda ctx: bins)
        return SimpleNamespace(dim=dim, nx=n[0], ny=n[1], nz=n[2], nspecies=species, ctx=None,
                               tuning=lambda: dict(filter_passes=passes))

    assert b.launches_per_step(sim(1, (512, 1, 1), 2, 0, 8)) == (2, 3 * 2 + 1)
    assert b.launches_per_step(sim(2, (1024, 1024, 1), 2, 0, 32768)) == (4, 5 * 2)
    assert b.launches_per_step(sim(3, (1024, 128, 128), 2, 4, 1 << 20), shock=True) == \
        (3 + 1 + 4 + 1, 5 * 2)
    # a small lattice with shock boundaries takes the separate field launches
    assert b.launches_per_step(sim(2, (48, 8, 1), 2, 0, 24), shock=True) == (3 + 1 + 1, 3 * 2)


def test_profiled_traffic_reads_the_summary_only_for_the_current_kernel(tmp_path, monkeypatch):
    b = _bench()
    h = b.kernel_source_hash()
    full = tmp_path / "full.md"
    full.write_text(f"text\n\n- kernel_source_hash: `{h}`\n- dram_bytes_per_full_launch: `1.5e9`\n")
    per = tmp_path / "per.md"
    per.write_text(f"- kernel_source_hash: `{h}`\n- dram_bytes_per_particle: `60.0`\n")
    stale = tmp_path / "stale.md"
    stale.write_text("- kernel_source_hash: `0000000000000000`\n- dram_bytes_per_particle: `60.0`\n")
    monkeypatch.setattr(b, "PROFILES", {"a": str(full), "b": str(per), "c": str(stale)})
    assert b.profiled_traffic("a", True, 123) == 1.5e9
    assert b.profiled_traffic("a", False, 123) is None  # a full-launch figure needs the full box
    assert b.profiled_traffic("b", False, 1000.0) == 60.0 * 1000.0
    assert b.profiled_traffic("c", True, 1000.0) is None  # taken on other kernel source
    assert b.profiled_traffic("missing", True, 1000.0) is None


def test_full_grid_of_each_workload():
    b = _bench()
    assert b.full_grid("turbulence_2d3v") == [1024, 1024]
    assert b.full_grid("weibel_1d3v") == [512]
    assert b.full_grid("shock_3d3v") == [1024, 128, 128]
    assert b.full_grid("shock_3d3v_periodic", 512) == [512, 64, 64]


def test_reference_line_carries_the_workload_config_and_the_contract_keys():
    import json
    import subprocess
    import sys

    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "3",
                        "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    b = _bench()
    assert d["impl"] == "reference" and d["metric"] == b.METRIC
    assert d["unit"] == "particle-steps/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["config"]["workload"] == "turbulence_2d3v"
    assert d["config"]["grid"] == [1024, 1024]  # the workload's, not the sample's
    assert "sample" in d["config"]
    cb = d["cpu_baseline"]
    # every host core, with the one-core figure beside it
    assert cb["kind"] == "oracle" and cb["cores"] == b.host_cores() and cb["value"] == d["value"]
    assert cb["single_core"]["cores"] == 1 and cb["single_core"]["value"] > 0
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
