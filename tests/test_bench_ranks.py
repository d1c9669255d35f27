"""Host logic of `bench.py --gpus N` on the CPU: N independent replicas (weak scaling, no
collective on the data path), a barrier around the timed region, the slowest rank's time, and
the whole job's rate = ranks x units per rank and step x steps / that time.  Two `gloo` ranks
stand in for two GPUs; the reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, ws: int, port: int, out: str):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        bench.barrier_ranks(ws)
        ms = [12.5, 20.0][rank]                     # rank 1 is the slower replica
        ms_max = bench.reduce_max_over_ranks(ms, ws, "cpu")
        bench.barrier_ranks(ws)
        rate = bench.whole_job_rate(ws, 1000.0, 40, ms_max)
        with open(f"{out}.{rank}", "w") as f:
            f.write(f"{ms_max} {rate}")
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time(tmp_path):
    out = str(tmp_path / "r")
    tmp.spawn(_rank, args=(2, _free_port(), out), nprocs=2, join=True)
    for r in range(2):
        ms_max, rate = (float(v) for v in open(f"{out}.{r}").read().split())
        assert ms_max == 20.0
        # 2 ranks x 1000 units x 40 steps in 20 ms
        assert rate == pytest.approx(2 * 1000 * 40 / 0.020, rel=1e-15)


def test_single_rank_needs_no_process_group():
    assert bench.reduce_max_over_ranks(3.25, 1, "cpu") == 3.25
    bench.barrier_ranks(1)
    assert bench.whole_job_rate(1, 8.0, 5, 10.0) == pytest.approx(4000.0)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
