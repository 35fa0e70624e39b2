"""Host logic of bench.py for N > 1 processes, on CPU with gloo: every rank
runs its own boxes (no data-path collective); the whole-job value is all
ranks' node updates over the slowest rank's time."""
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


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # uneven ranks: 1e9 updates in 2 s and 3e9 in 4 s
    updates = [1e9, 3e9][rank]
    seconds = [2.0, 4.0][rank]
    value, ms = bench.job_throughput(updates, seconds, world, torch.device("cpu"))
    q.put((rank, value, ms))
    dist.destroy_process_group()


def test_job_throughput_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms in res:
        assert ms == pytest.approx(4000.0)
        assert value == pytest.approx(4e9 / 4.0 / 1e6)


def test_job_throughput_single_process():
    import torch

    sys.path.insert(0, ROOT)
    import bench

    value, ms = bench.job_throughput(5e8, 0.5, 1, torch.device("cpu"))
    assert value == pytest.approx(1000.0) and ms == pytest.approx(500.0)


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
