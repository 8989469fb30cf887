"""Sharding of a sampling job over ranks (one process per GPU).

Shots are independent, and the output bits depend only on (circuit, seed,
global 64-shot chunk), so ranks need no exchange on the data path: rank r
samples its own contiguous range of global chunks and writes its own columns
of the detector-major output. Concatenating the ranks' columns in rank order
gives the single-GPU result bit for bit. The only collective is the
max-over-ranks reduction of the step time for reporting.
"""
from __future__ import annotations

from typing import Tuple


def rank_chunk_range(rank: int, world: int, shots_per_rank: int) -> Tuple[int, int]:
    """Weak scaling: every rank samples `shots_per_rank` shots; rank r starts
    at global chunk r * ceil(shots_per_rank / 64). Returns (first_chunk,
    shots). Ranks' chunk ranges are disjoint and contiguous in rank order."""
    if not (0 <= rank < world):
        raise ValueError("rank outside [0, world)")
    if shots_per_rank <= 0:
        raise ValueError("shots_per_rank must be positive")
    cols = (shots_per_rank + 63) // 64
    return rank * cols, shots_per_rank


def max_over_ranks(value: float, device=None) -> float:
    """Largest `value` over all ranks of the default process group (the
    value itself when torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
