"""The N > 1 path of the benchmark on the CPU (gloo, world size 2): every rank runs its own
replica of the step, and the whole-job throughput uses the slowest rank's time (a max over
ranks); no collective touches the solver's data."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        local_ms = 100.0 + 50.0 * rank  # the second replica is slower
        q.put((rank,) + bench.job_throughput(local_ms, 15, 5, world, dist, "cpu"))
    finally:
        dist.destroy_process_group()


def test_job_throughput_takes_the_slowest_rank_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(world))
    for rank, value, job_ms in out:
        assert job_ms == 150.0
        assert value == pytest.approx(15 * 5 * world / 0.150)


def test_job_throughput_single_rank_needs_no_process_group():
    import bench
    value, job_ms = bench.job_throughput(200.0, 15, 5, 1)
    assert job_ms == 200.0 and value == pytest.approx(15 * 5 / 0.2)
