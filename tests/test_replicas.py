"""The N > 1 path of bench.py (replicas under torchrun, one rank per GPU),
exercised on CPU: world size 2 over gloo.  The whole-job value is the units
all ranks processed over the slowest rank's time, and every rank agrees on
it; the reference arm runs on rank 0 only and the other ranks exit 0 without
work or output."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            init_method=f"tcp://127.0.0.1:{port}")
    import bench

    secs = [0.5, 0.8][rank]
    units = [100.0, 300.0][rank]
    t, v = bench.job_value(secs, units, dist)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"t": t, "v": v}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_job_value_is_all_units_over_the_slowest_rank(tmp_path):
    import torch.multiprocessing as mp

    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r in res:
        assert r["t"] == pytest.approx(0.8)
        assert r["v"] == pytest.approx(400.0 / 0.8)


def test_job_value_on_one_rank():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.job_value(2.0, 10.0) == (2.0, 5.0)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload",
                        "weibel_1d3v", "--steps", "3", "--warmup", "3", "--gpus", "2"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
    env = dict(os.environ, RANK="0", WORLD_SIZE="2", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload",
                        "weibel_1d3v", "--steps", "3", "--warmup", "3", "--gpus", "2"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
