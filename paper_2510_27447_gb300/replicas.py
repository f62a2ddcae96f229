"""Replica parallelism across GPUs.

The partitioned step of one simulation is not sharded here: every GPU runs
independent simulations (replicas) and no data crosses between them.  For a
multi-GPU measurement only the timing is combined: the work of all ranks
divided by the slowest rank's time (weak scaling).
"""
from __future__ import annotations


def whole_job_rate(local_units: float, local_seconds: float, device: str = "cpu"):
    """(sum of units over ranks / max seconds over ranks, max seconds).

    Works with any initialised torch.distributed backend (NCCL tensors on
    `device` = "cuda", gloo on "cpu"); without a process group it returns the
    local rate."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    secs = float(t.item())
    return float(u.item()) / secs, secs
