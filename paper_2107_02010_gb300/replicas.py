"""Whole-job figures of independent replicas.

One problem does not shard here, so `bench.py --gpus N` runs N independent
solves, one per rank, with no data-path collective; the only cross-rank step is
this reduction of the timing: the job takes as long as its slowest rank and
evaluates the pairs of all ranks.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def aggregate(t_total_s: float, pairs: float, device) -> tuple[float, float]:
    """(max over ranks of t_total_s, sum over ranks of pairs); identity on one rank."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(t_total_s), float(pairs)
    t = torch.tensor([t_total_s], dtype=torch.float64, device=device)
    p = torch.tensor([pairs], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t[0]), float(p[0])
