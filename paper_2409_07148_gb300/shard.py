"""Jump Restore chains across processes, one GPU each.

Chains are independent, and mu is state-independent (Alg. 2), so a chain set
splits into contiguous chain-id ranges, one per rank: the ranges give disjoint
Philox streams, and no shard has a start-up bias.  The only exchange is at
resolve: the estimator of Section 6.3 divides the sum of all splats by the
number J of completed tours, so the image over all ranks is the sum of the
ranks' accumulators divided by the sum of their J.  The collective is
torch.distributed's all_reduce (NCCL for CUDA tensors, gloo for CPU tensors).
"""
from __future__ import annotations


def chain_range(rank: int, world: int, n_total: int) -> tuple[int, int]:
    """(first chain id, chain count) of `rank` when n_total chains are split
    over `world` ranks as evenly as possible (the first n_total % world ranks
    take one more)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    if n_total < world:
        raise ValueError("fewer chains than ranks")
    base, extra = divmod(int(n_total), int(world))
    count = base + (1 if rank < extra else 0)
    first = rank * base + min(rank, extra)
    return first, count


def resolve_all(accum, tours: int, group=None):
    """Image over all ranks: accum is this rank's accumulator [H, W, 4]
    (RGB sums and the summed dt, float64 torch tensor on the collective's
    device), tours its J.  Reduces both in place over `group` and returns
    (image [H, W, 3], J over all ranks)."""
    import torch
    import torch.distributed as dist
    acc = accum if accum.dtype == torch.float64 else accum.double()
    dist.all_reduce(acc, op=dist.ReduceOp.SUM, group=group)
    j = torch.tensor([int(tours)], dtype=torch.float64, device=acc.device)
    dist.all_reduce(j, op=dist.ReduceOp.SUM, group=group)
    total = int(j.item())
    return acc[..., :3] / max(total, 1), total
