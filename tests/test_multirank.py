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


def _rank_lost(rank, world, port, q):
    import datetime
    import time

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        os._exit(3)  # this rank dies between steps, with no collective in flight
    import bench
    t0 = time.time()
    try:
        bench.job_throughput(100.0, 15, 5, world, dist, "cpu")
        q.put(("completed", time.time() - t0))
    except Exception as e:  # the lost peer surfaces as an error of the collective
        q.put((type(e).__name__, time.time() - t0))
    q.close()
    q.join_thread()  # the result is flushed before the hard exit
    os._exit(0)  # skip destroy_process_group: it would wait for the dead peer


def test_a_lost_rank_ends_the_max_over_ranks_with_an_error_gloo():
    """Failure detection on the host: when one rank dies, the others learn it from their next
    collective (the max over ranks of the timing), which fails within the process group's
    timeout instead of hanging."""
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_lost, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert procs[1].exitcode == 3 and procs[0].exitcode == 0
    what, waited = q.get(timeout=10)
    print("surviving rank saw:", what, f"after {waited:.1f} s")
    assert what != "completed" and waited < 60, (what, waited)


def _rank_shard(rank, world, port, q):
    """One rank of the sharded batch: it solves its own instances (tiny Lasso problems, solved
    here by the FP64 oracle as a CPU stand-in for the GPU batch), with no data exchange; the
    results are gathered afterwards only to check the partition."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import numpy as np

        import bench
        import gen
        import oracle
        n_inst = 9
        mine = bench.shard(n_inst, rank, world)
        solved = []
        for i in mine:
            D, y, _ = gen.lasso_problem(20, 40, seed=500 + i)
            lm, _, _ = oracle.lambda_max(D, y)
            solved.append((i, oracle.solve(D, y, 0.5 * lm, test="dst3", tol=1e-10, max_iter=20000)["x"]))
        local_ms = 10.0 * len(mine)
        value, job_ms = bench.job_throughput(local_ms, n_inst * 64 / world, 1, world, dist, "cpu")
        gathered = [None] * world
        dist.all_gather_object(gathered, solved)
        if rank == 0:
            q.put((gathered, value, job_ms))
    finally:
        dist.destroy_process_group()


def test_batch_instances_are_sharded_over_ranks_gloo():
    """Instance sharding of the batched workload on two gloo ranks: every instance is solved
    exactly once, on the rank bench.shard assigns it, the gathered results in instance order
    equal a single-rank run's, and the job time is the slowest rank's."""
    import numpy as np

    import bench
    import gen
    import oracle
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_shard, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered, value, job_ms = q.get(timeout=180)
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    ids = sorted(i for part in gathered for i, _ in part)
    assert ids == list(range(9))
    for r, part in enumerate(gathered):
        assert [i for i, _ in part] == bench.shard(9, r, world)
    by_id = {i: x for part in gathered for i, x in part}
    for i in range(9):
        D, y, _ = gen.lasso_problem(20, 40, seed=500 + i)
        lm, _, _ = oracle.lambda_max(D, y)
        np.testing.assert_array_equal(by_id[i], oracle.solve(D, y, 0.5 * lm, test="dst3", tol=1e-10,
                                                             max_iter=20000)["x"])
    assert job_ms == 50.0 and value == pytest.approx(9 * 64 / 0.050)
