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
