"""The multi-rank path of bench.py on CPU: two gloo ranks (no GPU).

The formation path has no exchange step, so N ranks run N replicas; what the
ranks share is the job's clock (the slowest rank's step time) and the
whole-job rate.  The reference arm runs on rank 0 alone."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, ms, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = bench.max_over_ranks(ms[rank], world, torch.device("cpu"))
        out[rank] = (m, bench.job_rate(world, 1000, m))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_the_slowest_time():
    world = 2
    ms = [3.0, 5.0]
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, _port(), ms, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    m, v = res[0]
    assert m == 5.0
    assert v == pytest.approx(2 * 1000 / 5e-3)


def test_one_rank_is_the_identity():
    assert bench.max_over_ranks(4.0, 1, None) == 4.0
    assert bench.job_rate(1, 10, 2.0) == pytest.approx(5000.0)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
