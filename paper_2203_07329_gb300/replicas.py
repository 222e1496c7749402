"""Bookkeeping for running independent replicas of the solver on N GPUs.

The method has no exchange step between GPUs: each rank solves its own set of
problems (or lambdas), so a multi-GPU run is N independent replicas (weak
scaling) and the only collectives are the timing barrier and the max-over-ranks
reduction of the step time.  Backend-agnostic (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


def env() -> tuple[int, int, int]:
    """(world_size, rank, local_rank) from the torchrun environment (1, 0, 0 without it)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def barrier(device: torch.device | None = None) -> None:
    if dist.is_available() and dist.is_initialized():
        dist.barrier()
    if device is not None and device.type == "cuda":
        torch.cuda.synchronize(device)


def max_over_ranks(value: float, device: torch.device | None = None) -> float:
    """The largest value over all ranks (the job's step time is its slowest rank's)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or torch.device("cpu"))
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, ms_per_step_max: float, world_size: int) -> float:
    """Whole-job units per second: every rank processes units_per_rank per step,
    and the step ends when the slowest rank ends."""
    return world_size * units_per_rank / (ms_per_step_max / 1e3)
