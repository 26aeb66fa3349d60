"""Spin sharding across ranks (§5.3.2 domain decomposition).

Spins are independent and the signal is additive over spin subsets (the file slave's
superposition, §5.3.2), so a multi-GPU run gives each rank a contiguous range of the object's
spins (strong scaling) or its own object of the same size (weak scaling) and exchanges exactly one
thing per step: the sum of the ranks' complex float64 signals.  Timing is the maximum over ranks.

Only host logic lives here (ranges, seeds, the reduction calls); the per-rank simulation is the
ordinary single-GPU path.  The helpers take an optional process group and work with any
torch.distributed backend (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

from typing import Optional, Tuple

SEED_STRIDE = 100  # seeds of weak-scaling ranks: base + SEED_STRIDE * rank + config id


def spin_range(n_spins: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous [start, stop) of the spins owned by `rank`; sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} of world {world}")
    if n_spins < 0:
        raise ValueError("n_spins < 0")
    q, r = divmod(n_spins, world)
    start = rank * q + min(rank, r)
    return start, start + q + (1 if rank < r else 0)


def shard_phantom(phantom, rank: int, world: int):
    """The rank's spins of a workloads.Phantom (strong scaling)."""
    import numpy as np

    a, b = spin_range(phantom.n, rank, world)
    return phantom.subset(np.arange(a, b))


def rank_seed(seed_base: int, config_id: int, rank: int) -> Optional[int]:
    """Seed of rank `rank`'s own object in a weak-scaling run (None = the config's default seed)."""
    return None if rank == 0 else seed_base + SEED_STRIDE * rank + config_id


def reduce_signal(signal, group=None) -> None:
    """Sum the ranks' signals in place (the one data exchange of a step)."""
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(signal, op=dist.ReduceOp.SUM, group=group)


def max_over_ranks(value: float, device=None, group=None) -> float:
    """Largest value over ranks (the step time of a multi-rank step)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
