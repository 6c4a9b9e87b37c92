"""The multi-rank bench logic on CPU with gloo (world size 2): ranks hash different streams of the
same size, the job time is the slowest rank's, and throughput counts every rank's bits."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 + 50.0 * rank
    t = bench.reduce_max(local_ms, world, "cpu")
    seed = bench.rank_stream_seed(3, rank)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, seed))


def test_two_rank_timing_and_sharding():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [150.0, 150.0]          # both ranks report the slowest time
    assert res[0][2] != res[1][2]                          # each rank hashes its own stream


def test_job_throughput_counts_all_ranks():
    import bench

    one = bench.job_throughput(1, 10**9, 10, 1000.0)
    assert one == pytest.approx(10.0)
    assert bench.job_throughput(4, 10**9, 10, 1000.0) == pytest.approx(4 * one)
