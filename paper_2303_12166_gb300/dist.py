"""Host-side helpers for running on several GPUs, one process per GPU.

The work of this library shards without any data-path exchange: independent
systems (a parameter sweep, served runs) are dealt to ranks, and a single
system is replicated (each rank advances its own copy).  Only the timing is
combined across ranks (the maximum).

A single system could also be split by element rows (`row_range`): each
rank advances its own rows with their accelerations against all N elements,
and the ranks all-gather positions and velocities once per step, after the
drift (the pair term needs every x_j, the contact test every v_j).  That
layout is exercised on CPU ranks with the FP64 reference; the library runs
one GPU per process.
"""
from __future__ import annotations


def shard(n_units: int, world: int, rank: int) -> list[int]:
    """Units of `rank` when n_units independent units are dealt round-robin
    over `world` ranks (every unit exactly once)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("need world >= 1 and 0 <= rank < world")
    return list(range(rank, n_units, world))


def row_range(n: int, world: int, rank: int) -> tuple[int, int]:
    """Rows [lo, hi) of `rank` when n element rows are split into `world`
    contiguous blocks whose sizes differ by at most one."""
    if world < 1 or not (0 <= rank < world) or n < 0:
        raise ValueError("need n >= 0, world >= 1 and 0 <= rank < world")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of `value` over the ranks of the default process group (the
    value itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
