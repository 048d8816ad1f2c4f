"""Serving loop: continuous batching of list-ranking and component jobs.

Jobs are submitted from any thread and return a :class:`concurrent.futures.Future`
that resolves to the result as a host ``numpy.int32`` array (ranks, or min-id
component labels). A scheduler thread runs the loop:

* admission  a launch unit is admitted once its jobs' device bytes (inputs and
             outputs) plus the growth of its stream's kernel workspace fit in
             the free part of the memory budget. The workspace a unit needs
             comes from the library (``workspace_query``); each stream's
             workspace is reserved through a library context before the unit
             is launched, and the bytes the context holds (``Context.bytes``)
             count against the budget. Admitted jobs keep their arrays resident
             on the device until they complete;
* batching   whenever a stream of the pool is idle, the jobs waiting at that
             moment form the next launch unit: up to ``max_batch`` small jobs of
             one kind (at most ``small_cutoff`` elements) are concatenated and
             ranked or labelled by one batched launch (``lr_rank_batched_sized``,
             ``cc_label_batched``); a larger job, or a small job that finds no
             other of its kind waiting, is launched alone (``lr_rank``,
             ``cc_label``);
* overlap    every unit runs on its own stream, so units admitted while others
             are on the GPU execute concurrently; inputs are copied in and
             results copied out on the unit's stream;
* completion events are polled; a finished unit's results are split per job,
             its memory is returned to the budget and its futures resolve.

Latency (submit to result on the host) and throughput are kept per job;
``stats()`` reports p50 / p99 latency and jobs per second.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import dataclasses
import threading
import time

import numpy as np
import torch

from . import (KIND_CC, KIND_CC_BATCH, KIND_LR, KIND_LR_BATCH, Context, cc_label, cc_label_batched, check,
               lr_rank, lr_rank_batched, workspace_query)

LIST, GRAPH = 0, 1


@dataclasses.dataclass
class Job:
    kind: int                        # LIST or GRAPH
    n: int                           # elements / vertices
    succ: torch.Tensor | None = None  # LIST: int32[n] host tensor (pinned is fastest)
    head: int = 0
    src: torch.Tensor | None = None   # GRAPH: int32[m] host tensors
    dst: torch.Tensor | None = None
    future: cf.Future | None = None
    t_submit: float = 0.0
    t_done: float = 0.0

    @property
    def m(self) -> int:
        return 0 if self.src is None else self.src.numel()

    def in_bytes(self) -> int:
        return 4 * (self.n if self.kind == LIST else 2 * self.m)

    def device_bytes(self) -> int:
        # resident arrays: inputs + output (kernel workspace is the stream's, counted apart)
        return self.in_bytes() + 4 * self.n


@dataclasses.dataclass
class _Unit:
    jobs: list
    stream: torch.cuda.Stream
    slot: int
    event: torch.cuda.Event
    out_host: torch.Tensor
    bytes: int
    keep: list


class Server:
    """Continuous-batching server on one GPU.

    mem_budget   device bytes the server may hold for resident job data
                 (default: half of the free device memory at start)
    streams      concurrent launch units
    small_cutoff jobs with at most this many elements are batched
    max_batch    jobs per batched launch
    """

    def __init__(self, device: int = 0, mem_budget: int | None = None, streams: int = 4,
                 small_cutoff: int = 1 << 18, max_batch: int = 512, out_cap: int = 1 << 26):
        self.device = torch.device("cuda", device)
        torch.cuda.set_device(self.device)
        free, _ = torch.cuda.mem_get_info(self.device)
        self.mem_budget = mem_budget if mem_budget is not None else free // 2
        self.small_cutoff = small_cutoff
        self.max_batch = max_batch
        self.out_cap = out_cap                     # elements of one unit's output
        self.streams = [torch.cuda.Stream(self.device) for _ in range(streams)]
        self.out_host = [torch.empty(out_cap, dtype=torch.int32).pin_memory() for _ in range(streams)]
        self.busy = [False] * streams
        self.ctx = Context(self.device.index if self.device.index is not None else 0)
        for st in self.streams:                    # the context adopts every stream's workspace
            self.ctx.reserve(st, 0)
        self.ws_bytes = self.ctx.bytes()           # bytes the library context holds (all streams)
        self.ws_cap = [0] * streams                # kernel workspace bytes each stream holds
        self.peak = self.ws_bytes                  # largest resident job bytes + workspace seen
        self.pending: collections.deque[Job] = collections.deque()
        self.inflight: list[_Unit] = []
        self.used = 0
        self.done: list[Job] = []
        self.lock = threading.Lock()
        self.wake = threading.Condition(self.lock)
        self.stop_flag = False
        self.t_first = None
        self.errors = 0
        self.cancelled = 0
        self.dead: BaseException | None = None   # why the scheduler stopped, if it failed
        self.thread = threading.Thread(target=self._loop, name="lrcc-serve", daemon=True)
        self.thread.start()

    # ------------------------------------------------------------ public
    def submit(self, job: Job) -> cf.Future:
        """Queue a job; the future resolves to its result. A job whose future is
        cancelled before it is launched is dropped."""
        if self.dead is not None:
            raise RuntimeError(f"serve: the scheduler stopped: {self.dead!r}")
        if job.device_bytes() > self.mem_budget or job.n > self.out_cap:
            raise ValueError("job larger than the server's memory budget or output buffer")
        job.future = cf.Future()
        job.t_submit = time.perf_counter()
        with self.lock:
            if self.t_first is None:
                self.t_first = job.t_submit
            self.pending.append(job)
            self.wake.notify()
        return job.future

    def submit_list(self, succ: torch.Tensor, head: int) -> cf.Future:
        return self.submit(Job(LIST, succ.numel(), succ=succ, head=int(head)))

    def submit_graph(self, src: torch.Tensor, dst: torch.Tensor, n: int) -> cf.Future:
        return self.submit(Job(GRAPH, int(n), src=src, dst=dst))

    def drain(self, timeout: float | None = None) -> None:
        t0 = time.perf_counter()
        while True:
            with self.lock:
                if not self.pending and not self.inflight:
                    return
            if timeout is not None and time.perf_counter() - t0 > timeout:
                raise TimeoutError("serve: drain timed out")
            time.sleep(0.0005)

    def close(self) -> None:
        with self.lock:
            self.stop_flag = True
            self.wake.notify()
        self.thread.join()
        self.ctx.close()

    def stats(self) -> dict:
        with self.lock:
            jobs = list(self.done)
        if not jobs:
            return {"jobs": 0}
        lat = np.array([j.t_done - j.t_submit for j in jobs]) * 1e3
        span = max(j.t_done for j in jobs) - min(j.t_submit for j in jobs)
        elems = sum(j.n + j.m for j in jobs)
        return {"jobs": len(jobs), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "jobs_per_s": len(jobs) / span, "melems_per_s": elems / span / 1e6,
                "errors": self.errors, "cancelled": self.cancelled, "workspace_bytes": self.ws_bytes,
                "peak_device_bytes": self.peak}

    # ---------------------------------------------------------- internals
    def _unit_ws(self, jobs: list) -> int:
        """Kernel workspace the library needs for this launch unit."""
        if len(jobs) == 1:
            j = jobs[0]
            return workspace_query(KIND_LR, j.n) if j.kind == LIST else workspace_query(KIND_CC, j.n, j.m)
        if jobs[0].kind == LIST:
            return workspace_query(KIND_LR_BATCH, sum(j.n for j in jobs), len(jobs))
        return workspace_query(KIND_CC_BATCH, sum(j.m for j in jobs), len(jobs))

    def _ws_growth(self, slot: int, need: int) -> int:
        # a workspace grows to at least 1.25x its size (the library's growth rule)
        old = self.ws_cap[slot]
        return 0 if need <= old else max(need, old + old // 4) - old

    def _take_unit(self, slot: int):
        """Pick the next launch unit for `slot` from the waiting jobs (lock held)."""
        if any(j.future.cancelled() for j in self.pending):
            kept = collections.deque(j for j in self.pending if not j.future.cancelled())
            self.cancelled += len(self.pending) - len(kept)
            self.pending = kept
        if not self.pending:
            return None
        first = self.pending[0]
        free = self.mem_budget - self.used - self.ws_bytes
        if first.n > self.small_cutoff:
            need = self._unit_ws([first])
            if first.device_bytes() + self._ws_growth(slot, need) > free:
                return None
            self.pending.popleft()
            return [first], need
        # a batch of small jobs of the first job's kind, in arrival order
        unit, bytes_, elems = [], 0, 0
        rest = collections.deque()
        while self.pending and len(unit) < self.max_batch:
            j = self.pending.popleft()
            if j.kind != first.kind or j.n > self.small_cutoff or bytes_ + j.device_bytes() > free \
                    or elems + j.n > self.out_cap:
                rest.append(j)
                if bytes_ + j.device_bytes() > free:
                    break
                continue
            unit.append(j)
            bytes_ += j.device_bytes()
            elems += j.n
        # leave jobs out (newest first) until the workspace growth fits as well
        need = self._unit_ws(unit) if unit else 0
        while unit and bytes_ + self._ws_growth(slot, need) > free:
            j = unit.pop()
            bytes_ -= j.device_bytes()
            rest.appendleft(j)
            need = self._unit_ws(unit) if unit else 0
        rest.extend(self.pending)
        self.pending = rest
        return (unit, need) if unit else None

    def _launch(self, jobs: list, slot: int, need: int) -> _Unit:
        stream = self.streams[slot]
        dev = self.device
        keep = []
        if need > self.ws_cap[slot]:
            # grow the stream's workspace through the context (the stream is idle)
            self.ctx.reserve(stream, need)
            held = self.ctx.bytes()
            with self.lock:
                self.ws_cap[slot] += held - self.ws_bytes
                self.ws_bytes = held
                self.peak = max(self.peak, self.used + self.ws_bytes)
        with torch.cuda.stream(stream):
            if len(jobs) == 1:
                # a job alone takes the single-instance call, which spreads it over
                # the whole GPU (the batched kernel gives each instance one block)
                j = jobs[0]
                out = torch.empty(j.n, dtype=torch.int32, device=dev)
                if j.kind == LIST:
                    s = j.succ.to(dev, non_blocking=True)
                    lr_rank(s, j.head, out=out, stream=stream)
                    keep += [s]
                else:
                    a = j.src.to(dev, non_blocking=True)
                    b = j.dst.to(dev, non_blocking=True)
                    cc_label(a, b, j.n, out=out, stream=stream)
                    keep += [a, b]
            elif jobs[0].kind == LIST:
                sizes = np.array([j.n for j in jobs], np.int64)
                off = np.zeros(len(jobs) + 1, np.int64)
                np.cumsum(sizes, out=off[1:])
                succ = torch.empty(int(off[-1]), dtype=torch.int32, device=dev)
                for j, b in zip(jobs, off[:-1]):
                    succ[b:b + j.n].copy_(j.succ, non_blocking=True)
                heads = torch.tensor([j.head for j in jobs], dtype=torch.int32).to(dev, non_blocking=True)
                offd = torch.from_numpy(off).to(dev, non_blocking=True)
                out = torch.empty(int(off[-1]), dtype=torch.int32, device=dev)
                lr_rank_batched(succ, offd, heads, out=out, stream=stream)
                keep += [succ, heads, offd]
            else:
                vs = np.array([j.n for j in jobs], np.int64)
                es = np.array([j.m for j in jobs], np.int64)
                voff = np.zeros(len(jobs) + 1, np.int64)
                eoff = np.zeros(len(jobs) + 1, np.int64)
                np.cumsum(vs, out=voff[1:])
                np.cumsum(es, out=eoff[1:])
                src = torch.empty(int(eoff[-1]), dtype=torch.int32, device=dev)
                dst = torch.empty(int(eoff[-1]), dtype=torch.int32, device=dev)
                for j, b in zip(jobs, eoff[:-1]):
                    src[b:b + j.m].copy_(j.src, non_blocking=True)
                    dst[b:b + j.m].copy_(j.dst, non_blocking=True)
                eo = torch.from_numpy(eoff).to(dev, non_blocking=True)
                vo = torch.from_numpy(voff).to(dev, non_blocking=True)
                out = torch.empty(int(voff[-1]), dtype=torch.int32, device=dev)
                cc_label_batched(src, dst, eo, vo, n_total=int(voff[-1]), out=out, stream=stream)
                keep += [src, dst, eo, vo]
            host = self.out_host[slot]
            host[: out.numel()].copy_(out, non_blocking=True)
            keep.append(out)
            ev = torch.cuda.Event()
            ev.record(stream)
        return _Unit(jobs, stream, slot, ev, host, sum(j.device_bytes() for j in jobs), keep)

    def _complete(self, u: _Unit) -> None:
        ok = True
        try:
            check(u.stream)
        except Exception as exc:          # device-detected error: fail the unit's jobs
            ok = False
            err = exc
        t = time.perf_counter()
        res = u.out_host.numpy()
        at = 0
        for j in u.jobs:
            j.t_done = t
            if ok:
                j.future.set_result(res[at:at + j.n].copy())
            else:
                j.future.set_exception(err)
            at += j.n
        held = self.ctx.bytes()   # a call may have grown its stream's workspace beyond the reservation
        with self.lock:
            self.ws_cap[u.slot] += held - self.ws_bytes
            self.ws_bytes = held
            self.peak = max(self.peak, self.used + self.ws_bytes)
            self.used -= u.bytes
            self.busy[u.slot] = False
            self.done.extend(u.jobs)
            if not ok:
                self.errors += len(u.jobs)

    def _loop(self) -> None:
        torch.cuda.set_device(self.device)
        try:
            self._run()
        except BaseException as exc:   # a failed scheduler fails every job it holds, never hangs them
            self._fail_all(exc)

    def _fail_all(self, exc: BaseException) -> None:
        with self.lock:
            self.dead = exc
            waiting = list(self.pending)
            running = [j for u in self.inflight for j in u.jobs]
            self.pending.clear()
            self.inflight = []
            self.errors += len(waiting) + len(running)
        err = RuntimeError(f"serve: the scheduler stopped: {exc!r}")
        for j in waiting:   # not started: a cancelled one stays cancelled
            if j.future.set_running_or_notify_cancel():
                j.t_done = time.perf_counter()
                j.future.set_exception(err)
        for j in running:
            if not j.future.done():
                j.t_done = time.perf_counter()
                j.future.set_exception(err)

    def _run(self) -> None:
        while True:
            # completions
            finished = [u for u in self.inflight if u.event.query()]
            for u in finished:
                self.inflight.remove(u)
                self._complete(u)
            with self.lock:
                if self.stop_flag and not self.pending and not self.inflight:
                    return
                launches = []
                for slot in range(len(self.streams)):
                    if self.busy[slot]:
                        continue
                    picked = self._take_unit(slot)
                    if picked is None:
                        break
                    jobs, need = picked
                    # a job cancelled since it was picked is dropped now; the others run
                    live = [j for j in jobs if j.future.set_running_or_notify_cancel()]
                    self.cancelled += len(jobs) - len(live)
                    if not live:
                        continue
                    if len(live) != len(jobs):
                        jobs, need = live, self._unit_ws(live)
                    self.busy[slot] = True
                    self.used += sum(j.device_bytes() for j in jobs)
                    self.peak = max(self.peak, self.used + self.ws_bytes)
                    launches.append((jobs, slot, need))
                if not launches and not self.inflight and not self.stop_flag:
                    self.wake.wait(timeout=0.01)
            for jobs, slot, need in launches:
                try:
                    self.inflight.append(self._launch(jobs, slot, need))
                except Exception as exc:
                    with self.lock:
                        self.busy[slot] = False
                        self.used -= sum(j.device_bytes() for j in jobs)
                        self.errors += len(jobs)
                    for j in jobs:
                        j.t_done = time.perf_counter()
                        j.future.set_exception(exc)
            if self.inflight and not launches:
                time.sleep(0.00005)


class FifoServer(Server):
    """Reference policy for comparison: one job at a time, one launch per job,
    one stream (no batching, no overlap)."""

    def __init__(self, device: int = 0, **kw):
        kw = dict(kw)
        kw["streams"] = 1
        kw["small_cutoff"] = 0
        super().__init__(device, **kw)
