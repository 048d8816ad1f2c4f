"""Replicas over several processes, one GPU each.

A single list or graph is not sharded: with N processes every rank runs its own
replica of the work, and nothing crosses ranks on the data path. What the ranks
share is the timing protocol: a barrier on both sides of the timed region and
the maximum of the per-rank times, from which the whole-job rate is the work of
all ranks divided by the slowest rank's time. The launcher (torchrun) gives each
process WORLD_SIZE, RANK, LOCAL_RANK and the rendezvous address.
"""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


def env() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the launcher's environment (1, 0, 0 alone)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str, device: torch.device | None = None) -> None:
    """Joins the process group when there is more than one rank (nccl binds `device`)."""
    world, _, _ = env()
    if world > 1 and not dist.is_initialized():
        if backend == "nccl":
            dist.init_process_group(backend, device_id=device)
        else:
            dist.init_process_group(backend)


def world_size() -> int:
    return dist.get_world_size() if dist.is_initialized() else 1


def barrier() -> None:
    if world_size() > 1:
        dist.barrier()


def max_over_ranks(x: float, device: torch.device) -> float:
    """The largest x over all ranks (x itself alone); `device` holds the reduction
    buffer: a CUDA device for nccl, the CPU for gloo."""
    if world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, ms_per_rank: float, device: torch.device) -> tuple[float, float]:
    """(whole-job units per second, the slowest rank's ms): every rank processed
    `units_per_rank` units; the job ends when the slowest rank does."""
    ms = max_over_ranks(ms_per_rank, device)
    return units_per_rank * world_size() / (ms / 1e3), ms


def shutdown() -> None:
    if dist.is_initialized():
        dist.destroy_process_group()
