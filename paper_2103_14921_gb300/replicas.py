"""Multi-GPU replicas: every rank solves its own problem, no data exchange on the solve path.

The only collective is on the host side of a measurement: the wall time of a
timed region is the maximum over ranks, and the throughput of the whole job is
the work of all ranks divided by that time.
"""
from __future__ import annotations

import os


def world():
    """``(world_size, rank, local_rank)`` from the launcher's environment (1, 0, 0 when absent)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of ``value`` over the ranks of the default process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, seconds_this_rank: float, device=None):
    """``(units per second of the whole job, max seconds)`` with weak scaling over the ranks."""
    import torch.distributed as dist
    ws = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    t = max_over_ranks(seconds_this_rank, device)
    return ws * units_per_rank / t, t
