"""Replica parallelism across GPUs (one process per GPU, no data-path collective).

The online phase shards by right-hand sides and by (model, frequency): every rank holds its own
factors and solves its own share; the only communication is the timing barrier and the
reduction of per-rank times and counts used for reporting.
"""
from __future__ import annotations

import os
from typing import List, Sequence, Tuple

import torch
import torch.distributed as dist


def env_ranks() -> Tuple[int, int, int]:
    """(world size, rank, local rank) from the launcher's environment (1, 0, 0 without one)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(items: Sequence, rank: int, world: int) -> List:
    """Contiguous, balanced share of ``items`` for ``rank`` (sizes differ by at most one)."""
    n = len(items)
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    hi = lo + q + (1 if rank < r else 0)
    return list(items[lo:hi])


def _device_for(backend: str) -> torch.device:
    return torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")


def max_over_ranks(x: float) -> float:
    """Maximum of a per-rank scalar (identity without a process group)."""
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device_for(dist.get_backend()))
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float) -> float:
    """Sum of a per-rank scalar (identity without a process group)."""
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device_for(dist.get_backend()))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier():
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def whole_job_rate(local_units: float, local_seconds: float) -> float:
    """Units processed by all ranks divided by the slowest rank's time."""
    return sum_over_ranks(local_units) / max_over_ranks(local_seconds)
