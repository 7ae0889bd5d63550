"""bench.py's multi-rank bookkeeping on world_size-2 gloo process groups (CPU).

Every rank steps its own replica of the workload (weak scaling, no data-path
collective); the job time is the slowest rank's and the job throughput sums
the ranks' points.
"""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 + 50.0 * rank            # rank 1 is the slow one
    slow = bench.max_over_ranks(local_ms, dist, "cpu")
    value = bench.job_throughput(524288, 10, world, slow)
    q.put((rank, slow, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_time_and_job_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slow, value in out:
        assert slow == pytest.approx(150.0)
        assert value == pytest.approx(524288 * 10 * 2 / 0.150 / 1e6)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_throughput(1_000_000, 2, 1, 1000.0) == pytest.approx(2.0)
