"""Multi-GPU layout of the method: independent replicas (weak scaling).

The library runs the method for one point set on one GPU, so several GPUs
serve as independent replicas: every rank (one process per GPU) owns an
independent point set of the same workload and runs the whole method on it;
the only collective is the timing reduction.  Host-side logic only (no
kernels here).
"""
from __future__ import annotations


def replica_seed(base_seed: int, rank: int) -> int:
    """Data seed of the point set a rank owns (rank 0 keeps the base seed)."""
    return base_seed + 7919 * rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest per-rank value (the job's step time is its slowest
    rank's); `dist` is torch.distributed or None for one process."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, points_per_rank: int, ms_per_step: float) -> float:
    """Points per second of the whole job: all ranks' points over the
    slowest rank's step time."""
    return world * points_per_rank / (ms_per_step / 1000.0)
