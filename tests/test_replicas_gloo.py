"""The N > 1 bench path (independent replicas, max-over-ranks timing) on CPU
with two gloo ranks."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    times = [1.0 + rank, 5.0 - rank, 2.0]
    got = bench.max_over_ranks(times, dist, "cpu")
    out.put((rank, got, bench.job_throughput(1000, world, got[0])))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_throughput():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, thr in res:
        assert got == [2.0, 5.0, 2.0]
        assert thr == pytest.approx(2000 / 2e-3 / 1e9)
