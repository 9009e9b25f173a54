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
