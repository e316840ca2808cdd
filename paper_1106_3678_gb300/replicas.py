"""Host-side logic of a multi-GPU run: one process per GPU, each solving its
own replica of the workload (the solve does not shard across GPUs, so there
is no data-path collective).  Only the timing is combined: every rank times
its own steps, the job's time is the maximum over ranks, and the whole-job
throughput is the number of solves all ranks completed divided by that
time.

The functions take the torch.distributed group implicitly (the default
group) and a device for the one-element tensors they exchange, so the same
code runs over NCCL on GPUs and over gloo on CPU (where it is tested).
"""
from __future__ import annotations

import os


def world() -> tuple[int, int, int]:
    """(world_size, rank, local_rank) from the launcher's environment."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, device=None) -> float:
    """The maximum of `value` over all ranks (the value itself when the job
    has one process or no process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    """The sum of `value` over all ranks."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(units_this_rank: float, seconds_this_rank: float, device=None) -> tuple[float, float]:
    """Whole-job throughput of replicas: (sum of units over ranks) / (max of
    seconds over ranks).  Returns (throughput, job_seconds)."""
    units = sum_over_ranks(units_this_rank, device)
    secs = max_over_ranks(seconds_this_rank, device)
    return units / secs if secs > 0 else float("nan"), secs
