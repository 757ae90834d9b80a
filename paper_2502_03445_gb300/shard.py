"""Sharding of independent reconstructions across ranks (one GPU each).

Bins (fixed-bit assignments of some qubits) and independent networks share
nothing, so the path is data-parallel with no exchange: each rank
reconstructs its own units, and only the timing is combined (the slowest
rank's time, the sum of units) -- weak scaling.  Units of uneven cost are
assigned by longest-processing-time-first so that the slowest rank is as
fast as possible."""
from __future__ import annotations

import heapq


def lpt_partition(costs, world_size: int):
    """Assign unit indices to ranks: largest cost first, to the currently
    least-loaded rank (ties to the lowest rank).  Returns a list per rank."""
    heap = [(0.0, r) for r in range(world_size)]
    heapq.heapify(heap)
    parts = [[] for _ in range(world_size)]
    for i in sorted(range(len(costs)), key=lambda k: (-costs[k], k)):
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(p) for p in parts]


def bins_for_rank(n_fixed: int, rank: int, world_size: int):
    """The fixed-bit assignments (integers < 2^n_fixed) reconstructed by
    `rank`: a round-robin share of all 2^n_fixed bins."""
    return list(range(rank, 1 << n_fixed, world_size))


def fixed_bits_of_bin(n_qubits: int, fixed_qubits, b: int):
    """Per-qubit fixed bits (0/1 list of length n_qubits) of bin `b`:
    bit i of b is the value of fixed_qubits[i]."""
    bits = [0] * n_qubits
    for i, q in enumerate(fixed_qubits):
        bits[q] = (b >> i) & 1
    return bits


def aggregate(local_units: float, local_seconds: float, dist=None, device=None):
    """(total units over ranks, slowest rank's seconds) -- the whole-job
    throughput is their ratio.  Without a process group the local values are
    returned."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return local_units, local_seconds
    import torch
    t = torch.tensor([local_seconds], dtype=torch.float64, device=device)
    u = torch.tensor([local_units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()), float(t.item())
