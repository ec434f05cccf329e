"""Multi-rank path of bench.py on CPU: two gloo ranks, each timing its own
replica; the job's time is the slowest rank's and its updates the sum."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, u = bench.aggregate_ranks(1.0 + rank, 1000 * (rank + 1), device="cpu")
    r, w = bench._dist()
    out.put((rank, t, u, r, w))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, t, u, r, w in res:
        assert t == 2.0 and u == 3000.0      # max time over ranks, sum of updates
        assert r == rank and w == 2


def test_single_process_aggregation_is_identity():
    import bench
    assert bench.aggregate_ranks(1.5, 42) == (1.5, 42.0)
