"""The multi-GPU form of the bench is independent replicas (the path does not
shard on one box): each rank times its own steps, the job's time is the
slowest rank's, and the throughput counts every rank's units.  The host side
of that -- max over ranks, whole-job throughput, rank 0 alone printing -- runs
here as two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench.dist_env()
        assert (r, w, lr) == (rank, world, rank)
        my_ms = 1000.0 + 250.0 * rank              # rank 1 is the slower replica
        dist.barrier()
        t = bench.max_over_ranks(my_ms, w)
        out[rank] = (t, bench.replica_throughput(10 * 3, w, t))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 1250.0
    # 30 units per rank, 2 ranks, 1.25 s: 48 units/s for the job
    assert res[0][1] == res[1][1] == pytest.approx(48.0)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.replica_throughput(10, 1, 500.0) == pytest.approx(20.0)


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun every rank starts bench.py --impl reference; ranks other
    than 0 exit 0 without work or output."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
