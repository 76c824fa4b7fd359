"""The multi-rank path of bench.py (independent replicas, max-over-ranks time)
on CPU with the gloo backend, world size 2."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    srcs = list(range(10, 20))
    mine = bench.rank_sources(srcs, rank)
    local_ms = [40.0, 55.0][rank]                       # rank 1 is the slowest
    gteps, tmax = bench.aggregate(local_ms, K=7, m=1_000_000, world=world, pg=dist, device="cpu")
    q.put((rank, mine, gteps, tmax))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
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
    (r0, s0, g0, t0), (r1, s1, g1, t1) = res
    assert t0 == t1 == 55.0                               # max over ranks
    assert abs(g0 - 2 * 7 * 1_000_000 / 0.055 / 1e9) < 1e-9 and g0 == g1
    assert s0[0] == 10 and s1[0] == 11 and sorted(s0) == sorted(s1)  # different starting sources
