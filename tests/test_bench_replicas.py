"""The N-replica path of bench.py on the host: two gloo ranks (CPU, no GPU)
run the barrier and max-over-ranks the timed blocks use, and the whole-job
rate counts every replica's cells over the slowest rank's time.  The
reference arm does its work on rank 0 alone."""

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sync = bench.ReplicaSync(dist, "cpu")
        sync.barrier()
        ms = [12.5, 20.0][rank]               # rank 1 is the slower replica
        worst = sync.max(ms)
        sync.barrier()
        q.put((rank, worst, bench.whole_job_rate(1000, 10, world, worst)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, worst, rate in got:
        assert worst == 20.0
        # 2 replicas x 1000 cells x 10 steps in 20 ms = 1 Mcell-updates/s
        assert rate == pytest.approx(1.0)


def test_one_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    sync = bench.ReplicaSync(None, "cpu")
    sync.barrier()
    assert sync.max(3.5) == 3.5
    assert bench.whole_job_rate(16777216, 20, 1, 14.2) == pytest.approx(
        16777216 * 20 / 14.2e-3 / 1e6)


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench
    # a rank other than 0 returns at once, before any oracle work
    assert bench.run_reference_arm(None, 1, 2) == 0
