"""The multi-GPU path of bench.py is replicas only: every rank solves its own
instance, the job time is the slowest rank's, and the value counts the
solves of all ranks.  Checked here with two gloo ranks on the CPU (no GPU):
the cross-rank maximum, the throughput formula, and that only rank 0 of the
reference arm prints."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=2)
    try:
        dev_ms, wall_ms = bench.reduce_max([100.0 + 50.0 * rank, 300.0 - 10.0 * rank], "cpu")
        dist.barrier()
        out[rank] = (dev_ms, wall_ms, bench.solves_per_hour(2, dist.get_world_size(), dev_ms))
    finally:
        dist.destroy_process_group()


def test_two_rank_max_and_throughput():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        dev_ms, wall_ms, v = res[rank]
        assert dev_ms == 150.0 and wall_ms == 300.0
        assert v == pytest.approx(3600.0 * 2 * 2 / 0.150)


def test_single_rank_reduce_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max([1.5, 2.5], "cpu") == [1.5, 2.5]
    assert bench.solves_per_hour(2, 1, 1000.0) == pytest.approx(7200.0)


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, env=env, cwd=ROOT, timeout=600)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_local_slopes_of_the_regimes_workload():
    """bench.local_slopes: a power law N^-a has log-log slope -a, and
    exp(-c sqrt N) has slope -c against sqrt N, between every pair."""
    import math
    import bench
    pts = [(n, n ** -0.6366) for n in (128, 256, 512, 1024)]
    assert all(abs(s + 0.6366) < 1e-12 for s in bench.local_slopes(pts, math.log))
    pts = [(n, math.exp(-3.5 * math.sqrt(n))) for n in (100, 400, 900)]
    assert all(abs(s + 3.5) < 1e-9 for s in bench.local_slopes(pts, math.sqrt))
