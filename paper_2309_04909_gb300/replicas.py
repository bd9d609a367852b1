"""Multi-GPU layout: one process per GPU, no data-path collective.

Every unit of the hot path (an element, a tensor, a request) is independent,
so N GPUs run N shards with no exchange between them.  Two layouts:
  weak    every rank processes its own batch of the same shape (own seed);
  strong  one batch of tensors is split across ranks, balanced by size
          (longest-processing-time greedy), each tensor whole on one rank.
The only collective is the timing reduction (max over ranks) and, in tests,
gathering results for comparison.
"""
from __future__ import annotations

import heapq
from typing import List, Sequence


def rank_seed(base: int, rank: int) -> int:
    """Seed of a rank's replica (weak scaling); distinct per rank."""
    return (base + 0x9E3779B97F4A7C15 * rank) & 0xFFFFFFFFFFFFFFFF


def shard_by_size(sizes: Sequence[int], world: int) -> List[List[int]]:
    """Split tensor indices over `world` ranks: largest first onto the least
    loaded rank.  Returns the index list of every rank (each sorted)."""
    heap = [(0, r) for r in range(world)]
    out: List[List[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(sizes)), key=lambda i: (-sizes[i], i)):
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + sizes[i], r))
    return [sorted(x) for x in out]


def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank scalar over the default process group (identity
    without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
