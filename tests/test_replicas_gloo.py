"""The multi-rank path of bench.py (replicas only: independent copies, no
data-path collective) with two gloo ranks on the CPU: whole-job time is the
slowest rank's, bytes are summed, and the reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    t, total, value = bench.aggregate(1.0 + rank, 100.0 * (rank + 1), world, "cpu")
    out.put((rank, t, total, value))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_max_time_sum_bytes_two_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, total, value in got:
        assert t == 2.0 and total == 300.0
        assert abs(value - 300.0 / 2.0 / 1e9) < 1e-18


def test_aggregate_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    t, total, value = bench.aggregate(0.5, 1e9, 1, "cpu")
    assert (t, total) == (0.5, 1e9) and abs(value - 2.0) < 1e-12


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
