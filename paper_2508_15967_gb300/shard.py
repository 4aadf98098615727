"""Data-parallel sharding of independent rays across processes (one per GPU).

Rays are independent (the paper's ensemble of independent problems, Sec. 5),
so forward tracing needs no communication: each rank traces a contiguous
sub-range, addressed in the C ABI by offset pointers with the full row stride.
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
