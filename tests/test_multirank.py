"""The multi-replica path of bench.py on CPU (gloo, world_size 2): every timestep's bound is independent,
so N GPUs run N replicas with no data exchange; the only collective is the maximum of the step times,
and the whole-job value counts every rank's units over the slowest rank's time."""
import os
import socket
import subprocess
import sys

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = bench.slowest_rank_ms(torch, dist, 10.0 + 5.0 * rank, "cpu")   # rank 1 is the slow replica
        q.put((rank, ms, bench.job_value(100, world, ms)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    assert [r[1] for r in res] == [15.0, 15.0]                       # both ranks see the max
    assert all(abs(r[2] - 100 * 2 / 0.015) < 1e-6 for r in res)     # every rank's units / slowest time


def test_single_rank_value():
    assert bench.slowest_rank_ms(torch, dist, 12.5, "cpu") == 12.5
    assert abs(bench.job_value(320, 1, 2.0) - 160000.0) < 1e-9


def test_reference_arm_other_ranks_exit_without_work():
    """Under torchrun the reference arm (the oracle on the host) runs on rank 0 only."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
