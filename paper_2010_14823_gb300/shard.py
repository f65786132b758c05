"""Multi-GPU layout: one process per GPU, each advancing its own domains.

Columns are independent (the paper's Section 2), so the path shards with no
exchange of data: under torchrun every rank generates and steps its own
domain (weak scaling: per-GPU work fixed as ranks are added).  The only
collectives are the timing barrier and the maximum of the elapsed times; no
collective touches the state.
"""
from __future__ import annotations

import os


def rank_env() -> tuple[int, int, int]:
    """(rank, world_size, local_rank) from the torchrun environment (defaults 0, 1, 0)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(base_seed: int, rank: int) -> int:
    """Each rank draws a distinct synthetic domain of the same recipe and size."""
    return base_seed + 7919 * rank


def column_range(ncols_total: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous column range of one rank when a single domain is split
    (strong scaling): sizes differ by at most one column."""
    q, r = divmod(ncols_total, world)
    start = rank * q + min(rank, r)
    return start, start + q + (1 if rank < r else 0)


def column_range_aligned(ncols_total: int, rank: int, world: int, align: int = 32) -> tuple[int, int]:
    """Contiguous column range of one part when a domain is split into
    `world` parts whose starts are multiples of `align` columns (a state view
    starting at such a column keeps the 256-byte alignment the step needs):
    whole blocks of `align` columns are shared out as evenly as possible and
    the last part ends at ncols_total.  Parts may be empty."""
    nblk = (ncols_total + align - 1) // align
    q, r = divmod(nblk, world)
    b0 = rank * q + min(rank, r)
    b1 = b0 + q + (1 if rank < r else 0)
    return min(b0 * align, ncols_total), min(b1 * align, ncols_total)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest value over all ranks (the job's time is its slowest rank's)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist=None, device=None) -> float:
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
