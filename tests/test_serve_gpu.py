"""Serving loop: every job's result is the same alone and in the mix (equal to
the oracle and to a single-instance call), with continuous batching, overlap
on several streams and admission under a tight memory budget."""
from __future__ import annotations

import random
import threading
import time

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1002_4482_gb300 as lrcc
from paper_1002_4482_gb300 import serve

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _make_jobs(count, seed, lo=6, hi=19):
    rng = random.Random(seed)
    sizes = gen.loguniform_sizes(count, lo, hi, seed)
    jobs = []
    for k, n in enumerate(sizes.tolist()):
        if rng.random() < 0.7:
            succ, head = gen.list_random(n, 1000 + k)
            jobs.append(("list", torch.from_numpy(succ).pin_memory(), head, oracle.lr_rank(succ, head)))
        else:
            src, dst = gen.er(n, 4 * n, 2000 + k)
            jobs.append(("graph", torch.from_numpy(src).pin_memory(), torch.from_numpy(dst).pin_memory(), n,
                         oracle.cc_uf(src, dst, n)))
    return jobs


def _run_mix(server, jobs, threads=2, seed=0):
    futs = [None] * len(jobs)

    def worker(idx):
        rng = random.Random(seed + idx)
        for i in range(idx, len(jobs), threads):
            j = jobs[i]
            if j[0] == "list":
                futs[i] = server.submit_list(j[1], j[2])
            else:
                futs[i] = server.submit_graph(j[1], j[2], j[3])
            time.sleep(rng.random() * 0.002)

    ts = [threading.Thread(target=worker, args=(t,)) for t in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    return [f.result(timeout=120) for f in futs]


def test_mix_matches_oracle_and_single_calls():
    jobs = _make_jobs(60, 1)
    srv = serve.Server(0, mem_budget=256 << 20, streams=3, small_cutoff=1 << 16, max_batch=64)
    try:
        results = _run_mix(srv, jobs)
        srv.drain(60)
        st = srv.stats()
    finally:
        srv.close()
    assert st["jobs"] == len(jobs) and st["errors"] == 0
    for j, r in zip(jobs, results):
        expect = j[3] if j[0] == "list" else j[4]
        assert np.array_equal(r, expect)
    # alone: the same jobs one by one through the single-instance calls
    for j, r in zip(jobs[:12], results[:12]):
        if j[0] == "list":
            single = lrcc.lr_rank(j[1].to(DEV), j[2]).cpu().numpy()
        else:
            single = lrcc.cc_label(j[1].to(DEV), j[2].to(DEV), j[3]).cpu().numpy()
        assert np.array_equal(r, single)


def test_admission_under_tiny_budget_and_fifo_reference():
    jobs = _make_jobs(30, 2, lo=8, hi=17)
    # a budget that holds only a few jobs at once: admission has to wait
    srv = serve.Server(0, mem_budget=24 << 20, streams=4, small_cutoff=1 << 12, max_batch=8)
    fifo = serve.FifoServer(0, mem_budget=24 << 20)
    try:
        a = _run_mix(srv, jobs, seed=5)
        b = _run_mix(fifo, jobs, seed=6)
    finally:
        srv.close()
        fifo.close()
    for j, x, y in zip(jobs, a, b):
        expect = j[3] if j[0] == "list" else j[4]
        assert np.array_equal(x, expect) and np.array_equal(y, expect)


def test_workspace_is_reserved_counted_and_freed_through_a_context():
    # the server reserves its streams' workspaces through a library context and
    # counts them against its budget; closing it frees them
    jobs = _make_jobs(24, 3, lo=12, hi=19)
    before = lrcc.workspace_bytes()
    budget = 96 << 20
    srv = serve.Server(0, mem_budget=budget, streams=2, small_cutoff=1 << 14, max_batch=16)
    try:
        results = _run_mix(srv, jobs, seed=9)
        srv.drain(60)
        st = srv.stats()
        held = srv.ctx.bytes()
    finally:
        srv.close()
    for j, r in zip(jobs, results):
        assert np.array_equal(r, j[3] if j[0] == "list" else j[4])
    assert st["workspace_bytes"] == held and held > 0
    assert st["peak_device_bytes"] <= budget
    assert lrcc.workspace_bytes() == before


def test_cancelled_jobs_are_dropped():
    # a budget that holds one job at a time, so later jobs wait; the cancelled
    # ones never run and the others still give their exact results
    jobs = _make_jobs(16, 4, lo=15, hi=16)
    srv = serve.Server(0, mem_budget=6 << 20, streams=1, small_cutoff=0)
    try:
        futs = [srv.submit_list(j[1], j[2]) if j[0] == "list" else srv.submit_graph(j[1], j[2], j[3]) for j in jobs]
        dropped = [i for i in range(4, 16, 3) if futs[i].cancel()]
        for i, (j, f) in enumerate(zip(jobs, futs)):
            if i in dropped:
                assert f.cancelled()
            else:
                assert np.array_equal(f.result(timeout=60), j[3] if j[0] == "list" else j[4])
        srv.drain(60)
        assert srv.stats()["cancelled"] == len(dropped)
    finally:
        srv.close()


def test_failed_scheduler_fails_its_jobs_instead_of_hanging():
    # a fault on the host inside the scheduler (injected by replacing its unit
    # choice): every job it holds fails at once, and later submits are refused
    srv = serve.Server(0, streams=2)
    try:
        def broken(slot):
            raise RuntimeError("injected scheduler fault")
        srv._take_unit = broken
        succ, head = gen.list_random(10_000, 7)
        f = srv.submit_list(torch.from_numpy(succ).pin_memory(), head)
        with pytest.raises(RuntimeError, match="scheduler stopped"):
            f.result(timeout=30)
        with pytest.raises(RuntimeError, match="scheduler stopped"):
            srv.submit_list(torch.from_numpy(succ).pin_memory(), head)
    finally:
        srv.close()


def test_allocation_failure_fails_its_unit_only():
    # the library's next workspace allocation fails (host-side injection): the job
    # that needed it fails with ERR_NOMEM, and the server goes on with the next one
    srv = serve.Server(0, streams=1, small_cutoff=0)
    try:
        succ, head = gen.list_random(1 << 20, 8)
        lrcc.debug_fail_allocs(1)
        f_bad = srv.submit_list(torch.from_numpy(succ).pin_memory(), head)
        with pytest.raises(lrcc.LrccError) as e:
            f_bad.result(timeout=60)
        assert e.value.status == lrcc.ERR_NOMEM
        f_ok = srv.submit_list(torch.from_numpy(succ).pin_memory(), head)
        assert np.array_equal(f_ok.result(timeout=60), oracle.lr_rank(succ, head))
    finally:
        lrcc.debug_fail_allocs(0)
        srv.close()


def test_invalid_job_fails_only_its_unit():
    srv = serve.Server(0, streams=2, small_cutoff=1 << 10)
    try:
        succ, head = gen.list_random(50_000, 3)
        bad = succ.copy()
        bad[int(np.flatnonzero(bad == -1)[0])] = head          # a cycle
        f_bad = srv.submit_list(torch.from_numpy(bad).pin_memory(), head)
        srv.drain(60)
        f_ok = srv.submit_list(torch.from_numpy(succ).pin_memory(), head)
        with pytest.raises(lrcc.LrccError):
            f_bad.result(timeout=60)
        assert np.array_equal(f_ok.result(timeout=60), oracle.lr_rank(succ, head))
    finally:
        srv.close()


def test_oversized_job_is_refused():
    srv = serve.Server(0, mem_budget=1 << 20, streams=1)
    try:
        with pytest.raises(ValueError):
            srv.submit_list(torch.zeros(1 << 20, dtype=torch.int32), 0)
    finally:
        srv.close()
