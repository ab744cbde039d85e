"""The multi-replica aggregation of bench.py on CPU: two gloo ranks.

Every rank runs its own replica and reports its own units and time; the job
throughput is the units of all ranks over the slowest rank's time, the same
number on every rank.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        units = [3.0e9, 5.0e9][rank]          # bases each replica spelled
        secs = [0.010, 0.025][rank]          # each replica's time
        bench.rank_barrier(world)
        out = {"max": bench.max_over_ranks(secs, world), "sum": bench.sum_over_ranks(units, world),
               "rate": bench.job_rate(units, secs, world)}
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        assert res[r]["max"] == pytest.approx(0.025)
        assert res[r]["sum"] == pytest.approx(8.0e9)
        assert res[r]["rate"] == pytest.approx(8.0e9 / 0.025)


def test_one_rank_is_identity():
    import bench
    assert bench.max_over_ranks(2.5, 1) == 2.5
    assert bench.sum_over_ranks(7.0, 1) == 7.0
    assert bench.job_rate(10.0, 2.0, 1) == 5.0


def _dead_rank_worker(rank, world, port, q):
    import datetime
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    import bench
    bench.rank_barrier(world)                 # step 1: both ranks
    if rank == 1:
        os._exit(0)                           # rank 1 leaves between steps, without a word
    try:
        bench.rank_barrier(world)             # step 2: the other rank is gone
        q.put((rank, "returned"))
    except Exception as e:                    # the process group reports it instead of hanging
        q.put((rank, type(e).__name__))
    q.close()
    q.join_thread()                           # the message is out before the process ends
    os._exit(0)


def test_dead_rank_ends_in_an_error_not_a_hang():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dead_rank_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    rank, outcome = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert rank == 0 and outcome != "returned"
