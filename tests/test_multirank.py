"""Multi-GPU path of the benchmark (replicas only, weak scaling) on CPU ranks.

Two gloo ranks check the whole-job aggregation the benchmark uses: the time is
the slowest rank's, the updates are the sum over ranks; ranks draw distinct
seeds (independent replicas, no data-path collective); the reference arm runs
on rank 0 only; a rank that fails between steps is detected by the survivor's
next collective (short process-group timeout), not by a hang."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 100.0 + 50.0 * rank
        t, u = bench.aggregate_ranks(local_ms, 1000 * (rank + 1), dist, device="cpu")
        q.put((rank, t, u, bench.rank_seeds(rank)))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=5) for _ in range(world))
    for rank, t, u, seeds in res:
        assert t == 150.0            # max over ranks
        assert u == 1000 + 2000      # sum over ranks
    assert set(res[0][3]).isdisjoint(res[1][3])   # independent replicas per rank


def _worker_dies(rank, world, port, q):
    """Rank 1 fails between steps (raises before the step's aggregation); rank 0
    must get an error from its next collective within the short process-group
    timeout instead of waiting forever."""
    import datetime
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        raise RuntimeError("rank 1 failed before the step's aggregation")
    try:
        bench.aggregate_ranks(100.0, 1000, dist, device="cpu")
        q.put((rank, "no error"))
    except Exception as e:  # the collective's error is the detection
        q.put((rank, type(e).__name__))


def test_failed_rank_is_detected_by_the_next_collective():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker_dies, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert procs[1].exitcode != 0            # the failing rank ended with its exception
    assert procs[0].exitcode is not None     # the survivor did not hang
    rank, outcome = q.get(timeout=5)
    assert rank == 0 and outcome != "no error"


def test_single_process_aggregation_is_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(12.5, 77, None) == (12.5, 77)


def test_reference_arm_other_ranks_exit_quietly(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup, gpus = 1, 0, 2
    bench.run_reference(A(), rank=1)
    assert capsys.readouterr().out == ""


def test_all_cores_oracle_sample_matches_single_process():
    """The all-cores CPU baseline runs the unmodified oracle in spawned processes, one
    replica each: its update count is the single-process sample's times the process
    count, and every process computes (replica r of each job) independently."""
    sys.path.insert(0, ROOT)
    import bench
    from oracle import oracle as orc
    orc.build()
    u1, t1 = bench.oracle_sample(3)
    u2, w2 = bench.oracle_sample_all_cores(3, 2)
    assert u2 == 2 * u1 and t1 > 0 and w2 > 0
