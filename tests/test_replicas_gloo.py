"""The N > 1 path of the benchmark on CPU: replicas with no data-path
collective, whose whole-job value is the steps of all ranks over the slowest
rank's time (world_size 2, gloo); and the reference arm's non-zero ranks,
which exit without work."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_local = 2.0 + rank            # rank 1 is the slower replica
    value, t = bench.replica_throughput(t_local, steps=10, dist=dist, device="cpu")
    out[rank] = (value, t)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_is_steps_of_all_ranks_over_the_slowest():
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        value, t = res[r]
        assert t == 3.0                       # the slower rank's time on both ranks
        assert abs(value - 2 * 10 / 3.0) < 1e-12


def test_single_rank_throughput_without_a_process_group():
    import bench
    value, t = bench.replica_throughput(4.0, steps=8)
    assert t == 4.0 and value == 2.0


def test_reference_arm_non_zero_rank_exits_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--lags", "2"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
