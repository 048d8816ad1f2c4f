"""The multi-process path on the CPU: two ranks over gloo, as bench.py runs N
replicas (one process per GPU) under torchrun. Each rank runs its own replica of
a small list ranking (here the oracle stands in for the GPU work), the ranks
line up on a barrier and the job time is the slowest rank's."""
from __future__ import annotations

import os
import socket
import time

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import gen
import oracle
from paper_1002_4482_gb300 import ranks


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica(rank: int, world: int, port: int, out: str) -> None:
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    assert ranks.env() == (world, rank, rank)
    ranks.init("gloo")
    assert ranks.world_size() == world
    cpu = torch.device("cpu")
    # each rank's replica: the same workload, seeded by nothing rank-specific
    succ, head = gen.list_random(20_000, 3)
    ranks.barrier()
    t0 = time.perf_counter()
    r = oracle.lr_rank(succ, head)
    if rank == 1:
        time.sleep(0.2)               # the slow rank sets the job time
    ms = (time.perf_counter() - t0) * 1e3
    ranks.barrier()
    rate, slowest = ranks.job_rate(len(succ), ms, cpu)
    assert slowest >= 200.0 and slowest >= ms
    assert rate == pytest.approx(len(succ) * world / (slowest / 1e3))
    assert ranks.max_over_ranks(float(rank), cpu) == world - 1
    assert r[head] == len(succ) - 1
    with open(f"{out}.{rank}", "w") as f:
        f.write(f"{slowest} {rate}\n")
    ranks.shutdown()


def test_two_replicas_over_gloo(tmp_path):
    world = 2
    out = str(tmp_path / "rank")
    mp.spawn(_replica, args=(world, _free_port(), out), nprocs=world, join=True)
    vals = [open(f"{out}.{r}").read().split() for r in range(world)]
    # every rank computed the same job time and rate
    assert vals[0] == vals[1]


def test_single_process_is_a_world_of_one():
    assert ranks.world_size() == 1
    assert ranks.max_over_ranks(3.5, torch.device("cpu")) == 3.5
    rate, ms = ranks.job_rate(1000, 2.0, torch.device("cpu"))
    assert ms == 2.0 and rate == pytest.approx(500_000.0)
