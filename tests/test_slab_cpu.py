"""Host logic of the slab decomposition (Maksimova et al. 2021, Sec. 3.2) on
CPU: the slab ranges and owner table, and the ghost exchange between ring
neighbours over gloo with 1, 2 and 3 ranks (CPU tensors standing in for each
rank's exported boundary slabs)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2110_11398_gb300 import slab


@pytest.mark.parametrize("cpd,world,R", [(129, 8, 2), (13, 4, 2), (5, 2, 2), (9, 9, 1), (65, 1, 2), (14, 4, 3)])
def test_slab_ranges_cover_the_box_evenly(cpd, world, R):
    rs = slab.slab_ranges(cpd, world, R)
    assert len(rs) == world
    xs = [x0 + k for x0, n in rs for k in range(n)]
    assert xs == list(range(cpd))
    sizes = [n for _, n in rs]
    assert max(sizes) - min(sizes) <= 1 and min(sizes) >= R
    tab = slab.owner_table(cpd, rs)
    for r, (x0, n) in enumerate(rs):
        assert np.all(tab[x0:x0 + n] == r)


@pytest.mark.parametrize("cpd,world,R", [(7, 4, 2), (5, 3, 2), (3, 4, 1)])
def test_slab_ranges_reject_ranks_narrower_than_R(cpd, world, R):
    with pytest.raises(ValueError):
        slab.slab_ranges(cpd, world, R)


def _rank_exports(rank, R=2, cpd=5):
    """Deterministic stand-ins for rank's side-0 and side-1 exports."""
    ncell = R * cpd * cpd
    out = []
    for side in (0, 1):
        g = np.random.default_rng(100 * rank + side)
        n = 0 if (rank, side) == (1, 0) else int(g.integers(1, 40))     # one empty message
        counts = np.zeros(ncell, np.int32)
        np.add.at(counts, g.integers(0, ncell, n), 1)
        rec = g.standard_normal((n, 4)).astype(np.float32)
        out.append((torch.from_numpy(counts), torch.from_numpy(rec)))
    return out


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
        a, b = _rank_exports(rank)
        for _ in range(2):                                  # twice: the ring stays in step
            (lc, lr), (rc, rr) = slab.exchange_ghosts(a, b)
        P, S = slab.reduce_momentum({"momentum": [rank, 1.0, -rank], "abs_momentum": 2.0 * rank})
        q.put((rank, lc.numpy(), lr.numpy(), rc.numpy(), rr.numpy(), P, S))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_ghost_exchange_over_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=120) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, lc, lr, rc, rr, P, S in res:
        left, right = (rank - 1) % world, (rank + 1) % world
        exp_l = _rank_exports(left)[1]         # the left rank's last slabs
        exp_r = _rank_exports(right)[0]        # the right rank's first slabs
        assert np.array_equal(lc, exp_l[0].numpy()) and np.array_equal(lr, exp_l[1].numpy())
        assert np.array_equal(rc, exp_r[0].numpy()) and np.array_equal(rr, exp_r[1].numpy())
        assert P == [sum(range(world)), float(world), -sum(range(world))]
        assert S == 2.0 * sum(range(world))


def test_ghost_exchange_single_rank_is_its_own_neighbour():
    a, b = _rank_exports(0)
    fl, fr = slab.exchange_ghosts(a, b)
    assert fl is b and fr is a
