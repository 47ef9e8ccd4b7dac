"""Whole-job figures of the replicas run (`bench.py --gpus N` under torchrun).

The adaptive step of one instance is not sharded: N ranks run N independent
replicas of the workload, with no data-path collective.  The only exchange
is the final one: leaf updates summed over the ranks, and the time of the
slowest rank.
"""
from __future__ import annotations

from typing import Tuple


def aggregate(updates: float, seconds: float, device: str = "cpu") -> Tuple[float, float]:
    """(sum of `updates` over the ranks, max of `seconds` over the ranks); the
    local values when no process group is initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(updates), float(seconds)
    s = torch.tensor([float(updates)], dtype=torch.float64, device=device)
    m = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    return float(s.item()), float(m.item())
