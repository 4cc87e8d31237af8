"""The N > 1 path of bench.py (replicas, max-over-ranks time, summed units) on CPU with gloo."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, u = bench.reduce_over_ranks(1.0 + rank, 100.0 * (rank + 1), world)
    q.put((rank, t, u))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_reduce_over_ranks_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(world))
    for rank, t, u in res:
        assert t == 1.0 + (world - 1)           # slowest rank
        assert u == sum(100.0 * (r + 1) for r in range(world))


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_over_ranks(2.5, 7.0, 1) == (2.5, 7.0)
