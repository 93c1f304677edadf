"""Multi-GPU plumbing for the benchmark (one process per GPU).

The transfer path partitions into independent problems (requests; or targets, each of which
needs only the sources within its radius), so ranks never exchange data on the hot path.
Weak scaling: every rank serves its own seeded request stream of the single-GPU size; the
only collectives are the barrier and the reductions of the timing results below.
"""
from __future__ import annotations


def rank_seed(base_seed: int, rank: int) -> int:
    """seed of rank `rank`'s independent request stream"""
    return base_seed + 7919 * rank


def shard_indices(n: int, rank: int, world: int) -> list[int]:
    """round-robin split of n independent units: disjoint, covering, balanced within one"""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    return list(range(rank, n, world))


def aggregate(local_ms: float, local_points: int, group=None):
    """max of the per-rank step times and sum of the points mapped (torch.distributed);
    returns (max_ms, total_points, whole-job points per second)"""
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" \
        else torch.device("cpu")
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=dev)
    p = torch.tensor([int(local_points)], dtype=torch.int64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(p, op=dist.ReduceOp.SUM, group=group)
    max_ms, total = float(t.item()), int(p.item())
    return max_ms, total, total / (max_ms / 1e3)
