"""Data-parallel sharding of independent rays across processes (one per GPU).

Rays are independent (the paper's ensemble of independent problems, Sec. 5),
so forward tracing needs no communication: each rank traces a contiguous
sub-range, addressed in the C ABI by offset pointers with the full row stride
(a batch of media: contiguous media balanced on their ray counts).
The adjoint's parameter gradient is a sum over rays, so the one exchange of
the data-parallel backward is a sum of the per-rank gradients.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard_bounds(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous, balanced [lo, hi) of n rays for `rank` of `world` (sizes differ by <= 1)."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, n >= 0")
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def shard_media(offsets, rank: int, world: int) -> tuple[int, int]:
    """Contiguous media [m_lo, m_hi) of a batch for `rank` of `world`, balanced
    on ray counts: the cuts are the media at which the prefix sum of rays
    (offsets, n_media + 1 non-decreasing entries) first reaches k total /
    world, so every rank's ray count is within one medium's count of the
    ideal.  Rank r traces rays [offsets[m_lo], offsets[m_hi])."""
    import numpy as np
    off = np.asarray(offsets, dtype=np.int64)
    if off.ndim != 1 or off.size < 1 or off[0] != 0 or (np.diff(off) < 0).any():
        raise ValueError("offsets must start at 0 and be non-decreasing")
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need world >= 1 and 0 <= rank < world")
    n_media, total = off.size - 1, int(off[-1])

    def cut(k: int) -> int:
        if k <= 0:
            return 0
        if k >= world:
            return n_media
        # first medium boundary whose prefix count reaches k total / world (exact integer test)
        return int(np.searchsorted(off * world, k * total, side="left"))

    return cut(rank), cut(rank + 1)


def ray_share(scaling: str, n: int, rank: int, world: int) -> tuple[int, int, int]:
    """What one rank of a data-parallel run traces, as (seed shard, lo, hi):
    weak scaling gives every rank its own independent set of n rays (seed
    shard = rank, all of [0, n)); strong scaling splits one fixed set of n
    rays (seed shard 0) into balanced contiguous ranges (shard_bounds)."""
    if scaling == "weak":
        if world < 1 or not 0 <= rank < world or n < 0:
            raise ValueError("need world >= 1, 0 <= rank < world, n >= 0")
        return rank, 0, n
    if scaling == "strong":
        return (0, *shard_bounds(n, rank, world))
    raise ValueError(f"scaling must be 'weak' or 'strong', not {scaling!r}")


def media_share(scaling: str, offsets, rank: int, world: int) -> tuple[int, int, int]:
    """What one rank traces of a batch of media, as (seed shard, m_lo, m_hi):
    weak scaling gives every rank its own independent batch (seed shard =
    rank, every medium); strong scaling splits one fixed batch into
    contiguous media balanced on their ray counts (shard_media)."""
    if scaling == "weak":
        if world < 1 or not 0 <= rank < world:
            raise ValueError("need world >= 1 and 0 <= rank < world")
        return rank, 0, len(offsets) - 1
    if scaling == "strong":
        return (0, *shard_media(offsets, rank, world))
    raise ValueError(f"scaling must be 'weak' or 'strong', not {scaling!r}")


def allreduce_gradient(grad: torch.Tensor, group=None) -> torch.Tensor:
    """Sum a per-rank gradient (dL/dtheta of that rank's rays) over all ranks, in place."""
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(grad, op=dist.ReduceOp.SUM, group=group)
    return grad


def max_over_ranks(seconds: float, device="cpu", group=None) -> float:
    """The slowest rank's time (the job's time for a bulk-synchronous step)."""
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
