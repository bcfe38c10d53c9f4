"""Host side of the N-GPU runs: independent replicas, one process per GPU.

Every rank factorizes its own matrices (no data-path collective: the method's
units -- whole factorizations -- are independent); the job's time is the
slowest rank's, taken with a MAX all-reduce after a barrier, and the job's
throughput is the units of all ranks over that time (weak scaling).
"""
from __future__ import annotations

import os


def world() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def slowest_ms(ms: float, device=None) -> float:
    """The largest `ms` over all ranks (the local value with one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, slowest: float, nranks: int) -> float:
    """Units per second of the whole job: every rank's units over the
    slowest rank's milliseconds."""
    return nranks * units_per_rank * 1000.0 / slowest
