"""The N>1 path of the benchmark on CPU: world_size 2 over gloo.

The hashing path shards by independent inputs (replicas, no data exchange);
the only cross-rank step is taking the slowest rank's step time. Two gloo
ranks check that helper and the whole-job throughput arithmetic.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    times = [10.0 + rank, 20.0 - rank]          # rank 1 slower on the first, faster on the second
    got = bench.max_over_ranks(times, world)
    out[rank] = got
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == [11.0, 20.0] and out[1] == [11.0, 20.0]


def test_replica_throughput():
    import bench
    assert bench.replica_throughput(1 << 30, 1, 1000.0) == pytest.approx((1 << 30) / 1e9)
    assert bench.replica_throughput(1 << 30, 4, 1000.0) == pytest.approx(4 * (1 << 30) / 1e9)
    assert bench.max_over_ranks([1.5, 2.5], 1) == [1.5, 2.5]
