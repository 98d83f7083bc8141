"""Multi-rank host logic of bench.py on CPU with the gloo backend (2 ranks)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, units = bench.aggregate(100.0 + 50.0 * rank, 1000.0 * (rank + 1), dist)
        boxes = list(bench.shard(64, rank, world))
        q.put((rank, ms, units, boxes))
    finally:
        dist.destroy_process_group()


def test_aggregate_and_shard_two_ranks():
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
    for rank, ms, units, boxes in res:
        assert ms == 150.0              # slowest rank
        assert units == 3000.0          # all ranks' work
    assert res[0][3] + res[1][3] == list(range(64))


@pytest.mark.parametrize("n,world", [(64, 3), (5, 8), (0, 2), (7, 1)])
def test_shard_partitions(n, world):
    parts = [list(bench.shard(n, r, world)) for r in range(world)]
    flat = [i for p in parts for i in p]
    assert flat == list(range(n))
    assert max(map(len, parts)) - min(map(len, parts)) <= 1


def test_aggregate_single_process():
    assert bench.aggregate(12.5, 7.0, None) == (12.5, 7.0)
