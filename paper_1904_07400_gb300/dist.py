"""Host-side plumbing for running independent solves on several GPUs (one process per GPU).

The solve of one grid has no data-path collective here: several GPUs run replicas, and a
batch of independent grids is split across ranks before any GPU work.  The split is greedy
longest-processing-time (LPT) on the cost nx * ny * log2(P_x * P_y), the transform work of a
grid's solve.  Every rank computes the same split from the same list, so no exchange is
needed to agree on it.

Timing across ranks uses a barrier and the maximum over ranks of each rank's elapsed time.
These work with any torch.distributed backend (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import heapq
import math


def padded_period(n: int) -> int:
    """Smallest even 2^a 3^b >= 2n - 1 (the library's padding rule)."""
    p = max(2, 2 * n - 1)
    while True:
        q = p
        if q % 2 == 0:
            while q % 2 == 0:
                q //= 2
            while q % 3 == 0:
                q //= 3
            if q == 1:
                return p
        p += 1


def solve_cost(nx: int, ny: int) -> float:
    """Relative cost of one force solve: transform work nx ny log2(P_x P_y)."""
    return nx * ny * math.log2(padded_period(nx) * padded_period(ny))


def shard_lpt(costs: list[float], world: int) -> list[list[int]]:
    """Split item indices over `world` ranks, greedy LPT: items by decreasing cost (ties by
    index), each to the currently least-loaded rank (ties by rank).  Deterministic."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    shards: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        shards[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    for s in shards:
        s.sort()
    return shards


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    """Maximum of x over all ranks (x itself for one rank)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
