"""Multi-rank host logic on CPU (gloo, world size 2): bins and uneven units
are split without overlap or loss, the load is balanced, and the aggregate
(total units, slowest rank) is what the bench reports."""
import os
import socket

import numpy as np
import pytest

from paper_2502_03445_gb300 import shard


def test_lpt_partition_covers_and_balances():
    rng = np.random.Generator(np.random.PCG64(1))
    costs = list(rng.exponential(1.0, size=257))
    for ws in (1, 2, 3, 8):
        parts = shard.lpt_partition(costs, ws)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # LPT guarantee: makespan <= 4/3 of the optimum >= max(mean, largest unit)
        assert max(loads) <= (4 / 3) * max(sum(costs) / ws, max(costs)) + 1e-9


def test_bins_partition_and_fixed_bits():
    n_fixed = 5
    seen = []
    for r in range(3):
        seen += shard.bins_for_rank(n_fixed, r, 3)
    assert sorted(seen) == list(range(32))
    bits = shard.fixed_bits_of_bin(8, [1, 4, 6], 0b101)
    assert bits == [0, 1, 0, 0, 0, 0, 1, 0]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = shard.bins_for_rank(4, rank, world)
        secs = 0.5 + rank            # rank 1 is the slowest
        units, slowest = shard.aggregate(len(mine) * 1024.0, secs, dist)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        q.put((rank, units, slowest, gathered))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, units, slowest, gathered in res:
        assert units == 16 * 1024.0          # every bin counted once
        assert slowest == 1.5               # the slowest rank's time
        assert sorted(b for g in gathered for b in g) == list(range(16))
        assert not set(gathered[0]) & set(gathered[1])
