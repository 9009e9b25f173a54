"""The per-kernel microbenchmark runs through the library's own timers: it
reports every timed field kernel with its launch count, a positive time and
the algorithmic bytes of its grid."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,grid,keys", [("filter", (68, 19, 41), ["filter"]),
                                            ("fields", (64, 48, 1), ["b_half", "e_update"])])
def test_microbench_reports_each_kernel(kind, grid, keys):
    from paper_1906_06306_gb300 import microbench

    out = microbench.run(kind, grid, iters=4)
    cells = grid[0] * grid[1] * grid[2]
    assert out["cells"] == cells
    for k in keys:
        assert out[k]["launches"] == 4 and out[k]["us_per_launch"] > 0
        assert out[k]["alg_bytes"] == {"filter": 24, "b_half": 36, "e_update": 48}[k] * cells
