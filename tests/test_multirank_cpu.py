"""Replica bookkeeping of bench.py on two CPU ranks (gloo): barrier and max-over-ranks timing.

The path does not shard (one problem per GPU), so N GPUs run N independent replicas; the
only cross-rank operations are the barrier and the maximum of the step times."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank          # rank 1 is the slow replica
    dist.barrier()
    m = bench.max_over_ranks(ms, world)
    q.put((rank, m, bench.job_throughput(1000, world, m)))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]
    assert abs(res[0][2] - 2 * 1000 / 15e-3 / 1e9) < 1e-15


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_throughput(165636900, 1, 10.0) == pytest.approx(16.56369)
