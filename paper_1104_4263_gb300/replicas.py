"""Replicas across GPUs: the solver path does not shard (one grid's FFT product and
Krylov basis live on one GPU), so several GPUs run independent problems -- here one
incidence angle per rank on the same scatterer -- with no data exchange.  Only the
timing and the work counts are combined across ranks (host-side, any backend).
"""
from __future__ import annotations

import math


def angle_for_rank(rank: int, n_angles: int = 8) -> float:
    """Incidence angle psi_j = 2 pi j / n_angles of rank j (cycling when ranks > n_angles)."""
    return 2.0 * math.pi * (rank % n_angles) / n_angles


def combine(units: float, seconds: float, dist=None):
    """(total units over ranks, max seconds over ranks); identity without a process group."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(units), float(seconds)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    u = torch.tensor([float(units)], dtype=torch.float64, device=dev)
    s = torch.tensor([float(seconds)], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(s, op=dist.ReduceOp.MAX)
    return float(u.item()), float(s.item())


def throughput(units: float, seconds: float, dist=None) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    total, tmax = combine(units, seconds, dist)
    return total / tmax if tmax > 0 else 0.0
