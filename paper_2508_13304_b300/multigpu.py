"""Host logic of the multi-GPU benchmark path.

The projector path shards without any exchange: candidates (poses), views or
whole registration problems are independent units.  Each rank processes its
own units on its own GPU; the only collective is a MAX over ranks of the
timed region (and a barrier around it), so throughput is the units of all
ranks divided by the slowest rank's time.
"""
from __future__ import annotations


def shard(n_units: int, rank: int, world: int) -> range:
    """Contiguous, balanced share of n_units for this rank (sizes differ by at
    most one; empty when world > n_units for the last ranks)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank / world")
    base, extra = divmod(n_units, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """MAX of a per-rank float over all ranks (the local value without a
    process group)."""
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


def aggregate_rate(units_all_ranks: float, steps: int, max_total_ms: float) -> float:
    """Whole-job throughput: units of all ranks per second of the slowest rank."""
    return units_all_ranks * steps / (max_total_ms * 1e-3)
