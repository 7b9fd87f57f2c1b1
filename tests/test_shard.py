"""Film sharding over ranks (paper_1501_07293_b300.shard): the partition and the
world_size-2 gather / max on CPU with the gloo backend (no GPU)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1501_07293_b300 import inputs
from paper_1501_07293_b300.shard import film_cost, gather, max_over_ranks, partition


def test_partition_covers_every_film_once_and_balances():
    grids = [f.grid for f in inputs.film_batch()]
    for world in (1, 2, 3, 8):
        parts = partition(grids, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(grids)))
        loads = [sum(film_cost(grids[i]) for i in p) for p in parts]
        # greedy LPT: no rank above the mean by more than the costliest film
        assert max(loads) - sum(loads) / world <= max(film_cost(g) for g in grids)


def test_partition_edge_cases():
    assert partition([], 3) == [[], [], []]
    assert partition([(4, 4, 1)], 2) in ([[0], []], [[], [0]])
    with pytest.raises(ValueError):
        partition([(4, 4, 1)], 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, nfilms, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    grids = [(8 + 4 * i, 6 + i, 1 + i % 3) for i in range(nfilms)]
    idx = partition(grids, world)[rank]
    # each film's "result" is a function of its index (what its batch would return)
    local = np.array([[i, 10.0 * i, -i] for i in idx]).reshape(len(idx), 3)
    full = gather(local, idx, nfilms)
    t = max_over_ranks(1.5 + rank)
    out.put((rank, full.tolist(), t))
    dist.barrier()
    dist.destroy_process_group()


def test_gather_and_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world, nfilms = 2, 7
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, nfilms, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = np.array([[i, 10.0 * i, -i] for i in range(nfilms)], dtype=np.float64)
    for rank, full, t in res:
        assert np.array_equal(np.array(full), want)
        assert t == 2.5   # the slowest rank
