"""Weak-scaling bookkeeping of the benchmark across ranks (one GPU per rank).

Every rank computes its own molecule (no data exchange: the path shards by
molecule with no dependence between ranks).  The only collectives are the
timing barrier and these reductions: the job's time is the slowest rank's,
its work the sum of every rank's grid points.  Works on any
torch.distributed backend (NCCL on GPUs; gloo in the CPU tests).
"""
from __future__ import annotations


def rank_env():
    """(world size, rank, local rank) from the launcher's environment."""
    import os

    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def job_totals(seconds: float, points: float, device="cpu"):
    """(max seconds over ranks, sum of points over ranks); identity on one rank."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(seconds), float(points)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    n = torch.tensor([float(points)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), float(n.item())


def job_max(seconds: float, device="cpu") -> float:
    return job_totals(seconds, 0.0, device)[0]


def throughput(points_all_ranks: float, steps: int, seconds_max: float) -> float:
    """Whole-job points per second: every rank's points of every step over the slowest rank's time."""
    return points_all_ranks * steps / seconds_max
