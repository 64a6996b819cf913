"""The multi-rank path of bench.py on CPU: two gloo ranks, each a replica
with its own timings; every rank sees the maximum, and the reported value is
the work of all ranks divided by the slowest rank's time."""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(('127.0.0.1', 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ['MASTER_ADDR'] = '127.0.0.1'
    os.environ['MASTER_PORT'] = str(port)
    dist.init_process_group('gloo', rank=rank, world_size=world)
    import bench
    local = [100.0 + 50.0 * rank, 1000.0 - 10.0 * rank]     # E_loc ms, step ms
    mx = bench.max_over_ranks(local)
    q.put((rank, mx, bench.job_throughput(8192, world, mx[0])))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_max_and_sum_the_work():
    ctx = mp.get_context('spawn')
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, value in out:
        assert mx == [150.0, 1000.0]
        assert value == pytest.approx(2 * 8192 / 0.150)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks([3.0, 4.0]) == [3.0, 4.0]
    assert bench.job_throughput(10, 1, 1000.0) == 10.0
