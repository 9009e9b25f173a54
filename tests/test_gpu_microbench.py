"""bench.py --micro times the field kernels alone through the library's own
timers: every timed field kernel with its launch count, a positive time and
the algorithmic bytes of its grid."""
import os
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("kind,grid,keys", [("filter", (68, 19, 41), ["filter"]),
                                            ("fields", (64, 48, 1), ["b_half", "e_update"])])
def test_micro_mode_reports_each_kernel(kind, grid, keys):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench

    out = bench.micro_run(kind, grid, iters=4)
    cells = grid[0] * grid[1] * grid[2]
    assert out["cells"] == cells
    for k in keys:
        assert out[k]["launches"] == 4 and out[k]["us_per_launch"] > 0
        assert out[k]["alg_bytes"] == {"filter": 24, "b_half": 36, "e_update": 48}[k] * cells
