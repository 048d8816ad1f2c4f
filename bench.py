#!/usr/bin/env python
"""Throughput of list ranking + connected components on GB300.

One step = lr_rank on a random-layout list of 2^28 elements followed by
cc_label on an R-MAT graph with 2^24 vertices and 2^28 edges (the large
plain-instance workload); ``--workload small`` uses a 2^20-element list and a
uniform random graph with 2^20 vertices and 2^22 edges instead. The value is
(list elements + graph edges) per second over the timed steps, with the
inputs resident in HBM; ``e2e`` repeats the measurement with the inputs copied
from pinned host memory and the results copied back inside every step.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mine|reference]
Under torchrun every rank runs its own replica (the single instances do not
shard) and rank 0 prints one JSON line with the max step time over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LR Mnodes/s and CC Medges/s at 1 GB300, % of HBM roofline; batched vs per-launch"
UNIT = "M(list nodes + graph edges)/s"
# bytes per element that the first ruling-set level moves, by layout (plan.rs_level0)
LR_METHOD_FIRST = {1: 40, 2: 34, 3: 38}
LR_METHOD_NOTE = {
    1: "select 4 B read + 8 B written, walk 8 B read + 8 B written, expand 8 B read + 4 B written",
    2: "walk 4 B read + 5 B written, scatter 5 B read + 8 B written, placement 8 B read + 4 B written",
    3: "select 4 B read + 4 B written, walk 8 B read + 8 B written, expand 8 B read + 4 B written",
}

# ncu DRAM bytes of one first-level walk launch (rs_walk0c) at n = 2^28, random
# layout: dram__bytes_read.sum + dram__bytes_write.sum of a one-pass capture of
# `bench.py --case lr 28 readonly` (31.904 GB + 1.715 GB), and the hash of the walk's
# source it was taken from. Reported only while that source is unchanged.
NCU_WALK0 = {"walk_sha1": "ad857f9e5fb29d9560eb4f03edf1b7bf29185207", "bytes_per_launch": 31904185600 + 1715129344}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["mine", "reference"], default="mine")
    ap.add_argument("--workload", choices=["large", "small"], default="large")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-families", action="store_true")
    ap.add_argument("--no-sweep", action="store_true", help="skip the list-ranking size sweep")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-jobs", type=int, default=2000)
    ap.add_argument("--plain-launches", action="store_true",
                    help="launch kernels directly instead of replaying CUDA graphs (for profilers that cannot "
                         "see kernels inside graphs with conditional nodes)")
    ap.add_argument("--case", nargs="+", metavar="ARG",
                    help="run one library call on a seeded input for a profiler and exit: "
                         "lr LOG2 [inplace|readonly|split] | wyllie LOG2 | cc SCALE | batch LOG2COUNT")
    return ap.parse_args()


def run_case(argv):
    """One call of the library on a seeded input, for profilers (ncu), with
    plain launches so that the profiler sees every kernel; the result is checked
    (the list's closed form, the component invariants) before it exits 0.

        lr 26 [inplace|readonly|split]   lr_rank, random list of 2^26
        wyllie 24                        lr_rank_wyllie
        cc 22                            cc_label, R-MAT scale 22, edge factor 16, then the
                                         gather probe over the same edges
        batch 10                         2^10 mixed instances, both batched calls
    """
    import torch
    import gen
    from gen import workloads
    import paper_1002_4482_gb300 as lrcc
    what, log2 = argv[0], int(argv[1])
    variant = argv[2] if len(argv) > 2 else ""
    dev = torch.device("cuda:0")
    for kind in (lrcc.KIND_LR, lrcc.KIND_LR_WYLLIE, lrcc.KIND_CC, lrcc.KIND_CC_SPARSE, lrcc.KIND_LR_BATCH,
                 lrcc.KIND_CC_BATCH):
        lrcc.set_plan(kind, 0, 32, use_graphs=2)
    level0 = {"inplace": 1, "readonly": 2, "split": 3}
    if variant in level0:
        lrcc.set_plan(lrcc.KIND_LR, 0, 32, rs_level0=level0[variant])
    if what in ("lr", "wyllie"):
        succ, head, perm = gen.list_random(1 << log2, 3, with_perm=True)
        s = torch.from_numpy(succ).to(dev)
        fn = lrcc.lr_rank if what == "lr" else lrcc.lr_rank_wyllie
        rank = fn(s, head)
        lrcc.check()
        r = rank.cpu().numpy()
        assert np.array_equal(r[perm], np.arange((1 << log2) - 1, -1, -1, dtype=np.int32))
    elif what == "cc":
        src, dst, n = workloads.cc_rmat(log2, 16)
        sd, dd = torch.from_numpy(src).to(dev), torch.from_numpy(dst).to(dev)
        lab_d = lrcc.cc_label(sd, dd, n)
        lrcc.check()
        # the hook pass's traffic without the hooking, over the same edges (its ceiling)
        lrcc.gather_probe(sd, dd, lab_d)
        lrcc.check()
        lab = lab_d.cpu().numpy()
        assert np.array_equal(lab[src], lab[dst]) and (lab <= np.arange(n)).all()
        assert np.array_equal(lab[lab], lab)
        log("rounds", lrcc.last_stats()["rounds"])
    elif what == "batch":
        (succ, off, heads), (src, dst, eoff, voff) = workloads.batch(1 << log2)
        lrcc.lr_rank_batched(*(torch.from_numpy(x).to(dev) for x in (succ, off, heads)))
        lrcc.cc_label_batched(*(torch.from_numpy(x).to(dev) for x in (src, dst, eoff, voff)))
        lrcc.check()
    else:
        raise SystemExit(f"unknown case {what}")
    torch.cuda.synchronize()
    log("ok", what, log2, variant)


def workload(name):
    from gen import workloads
    if name == "large":
        t = time.time()
        succ, head = workloads.lr_random(28)
        src, dst, n_cc = workloads.cc_rmat(24, 16)
        log(f"inputs generated in {time.time() - t:.1f} s")
        cfg = {"workload": "lr_random_2p28+cc_rmat_s24_ef16",
               "lr": {"n": len(succ), "layout": "uniform random permutation", "seed": 3},
               "cc": {"n": n_cc, "m": len(src), "generator": "R-MAT (0.57, 0.19, 0.19, 0.05), ids permuted",
                      "seed": 4}}
    else:
        succ, head = workloads.lr_random(20)
        src, dst, n_cc = workloads.cc_er(20, 22)
        cfg = {"workload": "lr_random_2p20+cc_er_2p20_2p22",
               "lr": {"n": len(succ), "layout": "uniform random permutation", "seed": 1},
               "cc": {"n": n_cc, "m": len(src), "generator": "uniform endpoints", "seed": 2}}
    return succ, head, src, dst, n_cc, cfg


def cpu_sample(name, log2s=26):
    """Bounded sample of the workload for the oracle: a 2^log2s-element list and
    the first 2^log2s edges of the graph, the workload's 1:1 mix of list
    elements and edges (2^26: about 12 s of one Arm core)."""
    from gen import workloads
    import gen
    if name == "large":
        succ, head = gen.list_random(1 << log2s, 3)
        src, dst, n_cc = workloads.cc_rmat(24, 16)
        src, dst = src[: 1 << log2s].copy(), dst[: 1 << log2s].copy()
        desc = (f"oracle walk of a 2^{log2s}-element random-layout list + union-find over the first "
                f"2^{log2s} edges of the R-MAT scale-24 edge list (2^24 vertices)")
    else:
        succ, head = workloads.lr_random(20)
        src, dst, n_cc = workloads.cc_er(20, 22)
        desc = "oracle on the full small workload (2^20 list, 2^20/2^22 graph)"
    return succ, head, src, dst, n_cc, desc


def time_oracle(sample):
    import oracle
    succ, head, src, dst, n_cc, _ = sample
    t0 = time.perf_counter()
    oracle.lr_rank(succ, head)
    t1 = time.perf_counter()
    oracle.cc_uf(src, dst, n_cc)
    t2 = time.perf_counter()
    return t2 - t0, t1 - t0, t2 - t1


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except OSError:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def walk0_sha1(path):
    """Hash of the first-level walk's source (lr.cu from the read-only walk's
    section header up to the count scan that follows it)."""
    text = open(path).read()
    a = text.index("// ------------------------------------------------ level 0, read-only walk")
    b = text.index("// Exclusive scan of each bucket's row")
    return hashlib.sha1(text[a:b].encode()).hexdigest()


def run_reference(args):
    """The reference arm: the CPU oracle, as it stands, on a bounded sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # one step is a bounded sample, halved for every doubling of the run's
    # steps beyond 13, so that the whole run stays within a few minutes
    log2s = 26 - max(0, math.ceil(math.log2(max(1, args.steps + args.warmup) / 13)))
    sample = cpu_sample(args.workload, max(22, log2s))
    units = len(sample[0]) + len(sample[2])
    for _ in range(args.warmup):
        time_oracle(sample)
    t = [time_oracle(sample)[0] for _ in range(args.steps)]
    total = sum(t)
    value = units * args.steps / total / 1e6
    cfg = workload_config_only(args.workload)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample[5]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config_only(name):
    if name == "large":
        return {"workload": "lr_random_2p28+cc_rmat_s24_ef16", "lr": {"n": 1 << 28}, "cc": {"n": 1 << 24, "m": 1 << 28}}
    return {"workload": "lr_random_2p20+cc_er_2p20_2p22", "lr": {"n": 1 << 20}, "cc": {"n": 1 << 20, "m": 1 << 22}}


def random_gather_peak(torch, dev, stream, log2n=28):
    """Independent random 4-byte gathers per second from a 2^log2n array (the
    random-access ceiling the walk is measured against), in G/s."""
    with torch.cuda.stream(stream):
        a = torch.arange(1 << log2n, dtype=torch.int32, device=dev)
        idx = torch.randperm(1 << log2n, device=dev)
        out = torch.empty_like(a)
        for _ in range(2):
            torch.index_select(a, 0, idx, out=out)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            torch.index_select(a, 0, idx, out=out)
        e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1) / 3
    del a, idx, out
    torch.cuda.empty_cache()
    return (1 << log2n) / (ms / 1e3) / 1e9


def chase_peak(lrcc, torch, succ, stream, chain_logs=(19, 20, 21, 22, 23)):
    """Dependent 4-byte reads of the bench's own successor array per second, in
    G/s, from the library's chase probe (the first-level walk's load form, none
    of its work), best over a few chain counts, each reading about n successors;
    returns (rate, chains)."""
    n = succ.numel()
    best = (0.0, 0)
    for lc in chain_logs:
        chains = 1 << lc
        steps = max(1, (n + chains - 1) // chains)
        lrcc.chase_probe(succ, chains, steps, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(2):
                lrcc.chase_probe(succ, chains, steps, stream=stream)
            e1.record(stream)
        stream.synchronize()
        lrcc.check(stream)
        rate = chains * steps / (e0.elapsed_time(e1) / 2 / 1e3) / 1e9
        if rate > best[0]:
            best = (rate, chains)
    return best


def bench_lr_sweep(lrcc, torch, dev, stream, sizes=(16, 18, 20, 22, 24, 26, 28)):
    """List-ranking throughput against list size for the three first-level layouts
    (in-place 8-byte words, read-only walk with chunked records, split mark and
    local-rank arrays) and both list layouts (random, ordered = even splitters along
    the list): where the rate changes as the list outgrows L2 (the paper's
    "inflection", Sec. 3.2). The paper's own comparison, the 48-bit split arrays
    (16-bit marks, so fewer than 65,535 splitters) against the packed 64-bit words
    at the same spacing, is measured on the random layout as `paper48` / `paper64`."""
    import gen
    out = []
    base = {k: lrcc.get_plan(lrcc.KIND_LR, 1 << k) for k in sizes}

    def best_ms(s_d, head, r_d):
        lrcc.lr_rank(s_d, head, out=r_d, stream=stream)
        stream.synchronize()
        best = float("inf")
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            lrcc.lr_rank(s_d, head, out=r_d, stream=stream)
            b.record(stream)
            b.synchronize()
            best = min(best, a.elapsed_time(b))
        lrcc.check(stream)
        return best

    try:
        for lg in sizes:
            n = 1 << lg
            row = {"log2n": lg}
            d48 = base[lg]["rs_spacing0"]
            while (n + d48 - 1) // d48 >= 0xFFFF:
                d48 *= 2
            for layout in ("random", "ordered"):
                succ_h, head = gen.list_random(n, 100 + lg) if layout == "random" else gen.list_ordered(n)
                with torch.cuda.stream(stream):
                    s_d = torch.from_numpy(succ_h).to(dev)
                    r_d = torch.empty_like(s_d)
                variants = [("inplace", 1, base[lg]["rs_spacing0"]), ("readonly", 2, base[lg]["rs_spacing0"]),
                            ("split", 3, base[lg]["rs_spacing0"])]
                if layout == "random":
                    variants += [("paper48", 3, d48), ("paper64", 1, d48)]
                for name, l0, d0 in variants:
                    lrcc.set_plan(lrcc.KIND_LR, lg, lg, rs_level0=l0, rs_spacing0=d0)
                    row[f"{layout}_{name}_gnodes_per_s"] = n / best_ms(s_d, head, r_d) / 1e6
                if layout == "random":
                    row["paper48_spacing0"] = d48
                del s_d, r_d
            out.append(row)
    finally:
        for lg in sizes:
            lrcc.set_plan(lrcc.KIND_LR, lg, lg, rs_level0=base[lg]["rs_level0"],
                          rs_spacing0=base[lg]["rs_spacing0"])
    return out


def bench_small_configs(lrcc, torch, dev, stream, hbm, reps=20):
    """The two small configurations as legs of their own: list ranking of a
    2^20-element random list, and components of a uniform random graph with
    2^20 vertices and 2^22 edges. Both fit in L2, so a 256 MB buffer is written
    between timed calls (L2 flushed); each call is timed alone with CUDA events
    on the launching stream, median of `reps`. The CPU baseline is the oracle
    timed on the same full inputs on one host core."""
    import oracle
    from gen import workloads
    flush = torch.empty(64 << 20, dtype=torch.int32, device=dev)

    def timed(fn):
        fn()
        stream.synchronize()
        ts = []
        for _ in range(reps):
            with torch.cuda.stream(stream):
                flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        lrcc.check(stream)
        ts.sort()
        return ts[len(ts) // 2], ts[0]

    out = {}
    succ_h, head, perm = workloads.lr_random(20, with_perm=True)
    n = len(succ_h)
    with torch.cuda.stream(stream):
        s_d = torch.from_numpy(succ_h).to(dev)
        r_d = torch.empty_like(s_d)
    med, best = timed(lambda: lrcc.lr_rank(s_d, head, out=r_d, stream=stream))
    # the ranks against the layout's closed form (position k of the list has rank n - 1 - k)
    assert np.array_equal(r_d.cpu().numpy()[perm], np.arange(n - 1, -1, -1, dtype=np.int32))
    # the CPU baseline: the oracle timed on the same list (its result is not used here)
    t0 = time.perf_counter()
    oracle.lr_rank(succ_h, head)
    t_cpu = time.perf_counter() - t0
    out["lr_random_2p20"] = {
        "metric": "Mnodes/s", "value": n / med / 1e3, "ms_median": med, "ms_min": best,
        "roofline": {"bound": "hbm", "achieved": 8 * n / (med / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                     "frac": 8 * n / (med / 1e3) / 1e9 / hbm, "traffic": None,
                     "note": "problem bytes (4 B succ read + 4 B rank written per element) over the whole call; "
                             "the 4 MB list is launch- and latency-bound"},
        "cpu_baseline": {"value": n / t_cpu / 1e6, "unit": "Mnodes/s", "cores": 1, "kind": "oracle",
                         "sample": "the same 2^20-element list, whole"}}
    src_h, dst_h, nv = workloads.cc_er(20, 22)
    m = len(src_h)
    with torch.cuda.stream(stream):
        a_d = torch.from_numpy(src_h).to(dev)
        b_d = torch.from_numpy(dst_h).to(dev)
        l_d = torch.empty(nv, dtype=torch.int32, device=dev)
    med, best = timed(lambda: lrcc.cc_label(a_d, b_d, nv, out=l_d, stream=stream))
    t0 = time.perf_counter()
    oracle.cc_uf(src_h, dst_h, nv)
    t_cpu = time.perf_counter() - t0
    pbytes = 8 * m + 4 * nv
    out["cc_er_2p20_2p22"] = {
        "metric": "Medges/s", "value": m / med / 1e3, "ms_median": med, "ms_min": best,
        "rounds": lrcc.last_stats(stream)["rounds"],
        "roofline": {"bound": "hbm", "achieved": pbytes / (med / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                     "frac": pbytes / (med / 1e3) / 1e9 / hbm, "traffic": None,
                     "note": "problem bytes (8 B per edge read, 4 B per label written) over the whole call"},
        "cpu_baseline": {"value": m / t_cpu / 1e6, "unit": "Medges/s", "cores": 1, "kind": "oracle",
                         "sample": "the same graph, whole (union-find)"}}
    del flush, s_d, r_d, a_d, b_d, l_d
    return out


def bench_even_splitters(lrcc, torch, dev, stream, sizes=(16, 20, 24, 28)):
    """The paper's Table 3 on GB300 (Sec. 3.2): the same random-layout list
    ranked with random splitters and with a perfect set of even splitters (list
    positions 0, D, 2D, ...: every sublist exactly D elements), both through the
    in-place first level at the plan's spacing D."""
    import gen
    out = []
    base = {k: lrcc.get_plan(lrcc.KIND_LR, 1 << k) for k in sizes}

    def best_ms(fn):
        fn()
        stream.synchronize()
        best = float("inf")
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            best = min(best, a.elapsed_time(b))
        lrcc.check(stream)
        return best

    try:
        for lg in sizes:
            n = 1 << lg
            D = base[lg]["rs_spacing0"]
            succ_h, head, perm = gen.list_random(n, 100 + lg, with_perm=True)
            with torch.cuda.stream(stream):
                s_d = torch.from_numpy(succ_h).to(dev)
                r_d = torch.empty_like(s_d)
                even = torch.from_numpy(np.ascontiguousarray(perm[::D])).to(dev)
            lrcc.set_plan(lrcc.KIND_LR, lg, lg, rs_level0=1)
            t_rand = best_ms(lambda: lrcc.lr_rank(s_d, head, out=r_d, stream=stream))
            t_even = best_ms(lambda: lrcc.lr_rank_splitters(s_d, head, even, out=r_d, stream=stream))
            if int(r_d[head].item()) != n - 1:
                raise AssertionError("even splitters gave a wrong head rank")
            out.append({"log2n": lg, "spacing": D, "random_ms": t_rand, "even_ms": t_even,
                        "random_gnodes_per_s": n / t_rand / 1e6, "even_gnodes_per_s": n / t_even / 1e6,
                        "even_speedup": t_rand / t_even})
            del s_d, r_d, even
    finally:
        for lg in sizes:
            lrcc.set_plan(lrcc.KIND_LR, lg, lg, rs_level0=base[lg]["rs_level0"])
    return out


def bench_families(lrcc, torch, dev, stream, m=8_000_000):
    """The paper's component families (Sec. 4): collections of random lists, random
    trees of degree k and random graphs of edge density d, all with m edges; hook
    passes and time of the default rule (atomicMin hooking with the sample pass)
    against the Shiloach-Vishkin rounds (hook rule 4) and against a first pass
    that links the endpoints themselves (hook rule 5)."""
    import gen
    out = []
    cases = [("lists", 1, None)] + [("trees", k, None) for k in (2, 3, 5, 10, 20)] + \
            [("random", None, d) for d in (0.001, 0.01)]
    base = lrcc.get_plan(lrcc.KIND_CC, 1 << 20)
    for kind, k, d in cases:
        if kind == "lists":
            src, dst, n = gen.list_graph(8, m // 8 + 1, 61)
        elif kind == "trees":
            src, dst, n = gen.tree_graph(8, m // 8 + 1, k, 62)
        else:
            n = gen.density_vertices(m, d)
            src, dst = gen.er(n, m, 63)
        with torch.cuda.stream(stream):
            S = torch.from_numpy(src).to(dev)
            D = torch.from_numpy(dst).to(dev)
            lab = torch.empty(n, dtype=torch.int32, device=dev)
        row = {"family": kind, "k": k, "density": d, "n": n, "m": len(src)}
        ref = None
        for name, hook in (("atomicmin", base["cc_hook"]), ("shiloach_vishkin", 4), ("link_first_pass", 5)):
            lrcc.set_cc_plan(0, 32, cc_hook=hook)
            lrcc.cc_label(S, D, n, out=lab, stream=stream)
            stream.synchronize()
            best = float("inf")
            for _ in range(3):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                lrcc.cc_label(S, D, n, out=lab, stream=stream)
                b.record(stream)
                b.synchronize()
                best = min(best, a.elapsed_time(b))
            lrcc.check(stream)
            row[name] = {"ms": best, "rounds": lrcc.last_stats(stream)["rounds"]}
            if ref is None:
                ref = lab.clone()
            elif not torch.equal(ref, lab):
                raise AssertionError(f"hook rules disagree on {kind} {k} {d}")
        lrcc.reset_plans()
        row["sv_round_bound"] = int(math.floor(math.log(n) / math.log(1.5))) + 2
        out.append(row)
        del S, D, lab, ref
    return out


def bench_batched(lrcc, torch, dev, stream, log2_count=12, world=1, rank_id=0, max_fn=None):
    """4096 instances (2048 lists + 2048 graphs of average degree 4, sizes
    log-uniform in [2^8, 2^20)): one batched launch per kind against one
    launch per instance on the same stream, and spread over 8 streams. With
    several ranks the instances are shared out by LPT (shard.py) and every rank
    runs one batched launch per kind on its share; the time is the slowest
    rank's (the per-instance comparison runs alone only)."""
    from gen import workloads
    from paper_1002_4482_gb300 import shard
    (succ, off, heads), (src, dst, eoff, voff) = workloads.batch(1 << log2_count)
    all_units = len(succ) + len(src)
    if world > 1:
        li = shard.lpt_assign(shard.list_costs(off), world)[rank_id]
        gi = shard.lpt_assign(shard.graph_costs(eoff, voff), world)[rank_id]
        succ, off, heads = shard.list_share(succ, off, heads, li)
        src, dst, eoff, voff = shard.graph_share(src, dst, eoff, voff, gi)
    with torch.cuda.stream(stream):
        S, O, H = (torch.from_numpy(x).to(dev) for x in (succ, off, heads))
        SR, DS, EO, VO = (torch.from_numpy(x).to(dev) for x in (src, dst, eoff, voff))
        rank = torch.empty_like(S)
        lab = torch.empty(int(voff[-1]), dtype=torch.int32, device=dev)
    stream.synchronize()

    def ev(fn, reps):
        fn()
        stream.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        stream.synchronize()
        lrcc.check(stream)
        return a.elapsed_time(b) / reps

    lr_b = ev(lambda: lrcc.lr_rank_batched(S, O, H, out=rank, stream=stream), 3)
    cc_b = ev(lambda: lrcc.cc_label_batched(SR, DS, EO, VO, n_total=int(voff[-1]), out=lab, stream=stream), 3)
    if world > 1:
        slowest = max_fn(lr_b + cc_b)
        return {"workload": "2048 lists + 2048 graphs (avg degree 4), sizes log-uniform [2^8, 2^20), int64 offsets; "
                            f"instances shared out over {world} ranks by LPT, one batched launch per kind per rank",
                "ranks": world, "rank0_instances": {"lists": int(len(heads)), "graphs": int(len(voff) - 1)},
                "rank0_batched_ms": {"lr": lr_b, "cc": cc_b}, "slowest_rank_ms": slowest,
                "batched_melems_per_s": all_units / slowest / 1e3}
    offs, hs, eo, vo = off.tolist(), heads.tolist(), eoff.tolist(), voff.tolist()

    def per_lr():
        for k in range(len(hs)):
            lrcc.lr_rank(S[offs[k]:offs[k + 1]], hs[k], out=rank[offs[k]:offs[k + 1]], stream=stream)

    def per_cc():
        for k in range(len(vo) - 1):
            lrcc.cc_label(SR[eo[k]:eo[k + 1]], DS[eo[k]:eo[k + 1]], vo[k + 1] - vo[k],
                          out=lab[vo[k]:vo[k + 1]], stream=stream)

    lr_p = ev(per_lr, 1)
    cc_p = ev(per_cc, 1)

    # the same launches round-robin over 8 streams (each with its own workspace)
    side = [torch.cuda.Stream(device=dev) for _ in range(8)]

    def fanned(body):
        def run():
            e = torch.cuda.Event()
            e.record(stream)
            for s_ in side:
                s_.wait_event(e)
            body()
            for s_ in side:
                e = torch.cuda.Event()
                e.record(s_)
                stream.wait_event(e)
        return run

    def per_lr8():
        for k in range(len(hs)):
            lrcc.lr_rank(S[offs[k]:offs[k + 1]], hs[k], out=rank[offs[k]:offs[k + 1]], stream=side[k % 8])

    def per_cc8():
        for k in range(len(vo) - 1):
            lrcc.cc_label(SR[eo[k]:eo[k + 1]], DS[eo[k]:eo[k + 1]], vo[k + 1] - vo[k],
                          out=lab[vo[k]:vo[k + 1]], stream=side[k % 8])

    lr_p8 = ev(fanned(per_lr8), 1)
    cc_p8 = ev(fanned(per_cc8), 1)
    for s_ in side:
        lrcc.check(s_)
        lrcc.release(s_)
    units = len(succ) + len(src)
    return {"workload": "2048 lists + 2048 graphs (avg degree 4), sizes log-uniform [2^8, 2^20), int64 offsets",
            "list_nodes": int(len(succ)), "graph_vertices": int(voff[-1]), "graph_edges": int(len(src)),
            "batched_ms": {"lr": lr_b, "cc": cc_b, "total": lr_b + cc_b},
            "per_launch_ms": {"lr": lr_p, "cc": cc_p, "total": lr_p + cc_p},
            "per_launch_8_streams_ms": {"lr": lr_p8, "cc": cc_p8, "total": lr_p8 + cc_p8},
            "speedup": (lr_p + cc_p) / (lr_b + cc_b),
            "batched_melems_per_s": units / (lr_b + cc_b) / 1e3}


def bench_serve(torch, count=2000, seed=6, loads=(0.5, 0.8, 0.95), repeats=3):
    """Poisson stream of mixed jobs (70 % lists / 30 % graphs of average
    degree 8, sizes log-uniform in [2^10, 2^24)) through the continuous-
    batching server and through one-launch-per-job FIFO: saturated (all
    submitted at once) and at offered loads of 0.5, 0.8 and 0.95 times the
    batched server's saturated rate; every run `repeats` times, reported as the
    median with the range."""
    import gen
    from gen import workloads
    from paper_1002_4482_gb300 import serve
    # inputs come from a pool of seeded instances on an 8-per-octave size grid
    # (a job's size is rounded down to the grid), so the host builds them in seconds
    grid = np.unique(np.floor(2.0 ** np.arange(10, 24.01, 0.125)).astype(np.int64))
    _, kind, size = workloads.serve_jobs(count, 1.0, seed=seed)
    pool = {}

    def get(kd, n):
        g = int(grid[np.searchsorted(grid, n, side="right") - 1])
        if (kd, g) not in pool:
            if kd == 0:
                sc, h = gen.list_random(g, g)
                pool[(kd, g)] = (torch.from_numpy(sc).pin_memory(), h)
            else:
                a, b = gen.er(g, 4 * g, g)
                pool[(kd, g)] = (torch.from_numpy(a).pin_memory(), torch.from_numpy(b).pin_memory(), g)
        return pool[(kd, g)]

    jobs = [(int(k), get(int(k), int(n))) for k, n in zip(kind, size)]

    def run(srv, gaps):
        futs = []
        t = time.perf_counter()
        for (k, p), g in zip(jobs, gaps):
            t += g
            d = t - time.perf_counter()
            if d > 0:
                time.sleep(d)              # releases the GIL for the scheduler thread
            futs.append(srv.submit_list(p[0], p[1]) if k == 0 else srv.submit_graph(p[0], p[1], p[2]))
        for f in futs:
            f.result(timeout=600)
        st = srv.stats()
        srv.close()
        return st

    def summary(runs):
        out = {}
        for key in ("p50_ms", "p99_ms", "jobs_per_s"):
            v = sorted(r[key] for r in runs)
            out[key] = v[len(v) // 2]
            out[key + "_range"] = [v[0], v[-1]]
        return out

    res = {"workload": f"{count} jobs per run: 70 % lists / 30 % graphs (degree 8), sizes log-uniform [2^10, 2^24) "
                       "rounded down to an 8-per-octave grid of seeded pooled instances",
           "repeats": repeats, "saturated": {}, "loads": {}}
    sat = {"batched": [], "fifo": []}
    for _ in range(repeats):
        sat["batched"].append(run(serve.Server(0, streams=4), np.zeros(count)))
        sat["fifo"].append(run(serve.FifoServer(0), np.zeros(count)))
    res["saturated"] = {k: summary(v) for k, v in sat.items()}
    lam_sat = res["saturated"]["batched"]["jobs_per_s"]
    for load in loads:
        lam = load * lam_sat
        row = {"offered_jobs_per_s": lam, "batched": [], "fifo": []}
        for r in range(repeats):
            gaps = np.random.default_rng(seed * 100 + r).exponential(1.0 / lam, count)
            row["batched"].append(run(serve.Server(0, streams=4), gaps))
            row["fifo"].append(run(serve.FifoServer(0), gaps))
        res["loads"][str(load)] = {"offered_jobs_per_s": lam, "batched": summary(row["batched"]),
                                   "fifo": summary(row["fifo"])}
    return res


def main():
    args = parse()
    if args.case:
        run_case(args.case)
        return
    if args.warmup < 3:
        log("warmup raised to 3")
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return

    import torch

    import paper_1002_4482_gb300 as lrcc
    from paper_1002_4482_gb300 import ranks

    world, rank, local = ranks.env()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    ranks.init("nccl", dev)
    barrier = ranks.barrier

    def max_over_ranks(x):
        return ranks.max_over_ranks(x, dev)

    if args.plain_launches:
        for kind in (lrcc.KIND_LR, lrcc.KIND_LR_WYLLIE, lrcc.KIND_CC, lrcc.KIND_CC_SPARSE):
            lrcc.set_plan(kind, 0, 32, use_graphs=2)
    succ_h, head, src_h, dst_h, n_cc, cfg = workload(args.workload)
    n_lr, m_cc = len(succ_h), len(src_h)
    units = n_lr + m_cc
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        succ = torch.from_numpy(succ_h).to(dev)
        src = torch.from_numpy(src_h).to(dev)
        dst = torch.from_numpy(dst_h).to(dev)
        rank_out = torch.empty(n_lr, dtype=torch.int32, device=dev)
        label = torch.empty(n_cc, dtype=torch.int32, device=dev)
    stream.synchronize()

    def step():
        lrcc.lr_rank(succ, head, out=rank_out, stream=stream)
        lrcc.cc_label(src, dst, n_cc, out=label, stream=stream)

    # warm-up (also builds the graphs and the workspace); the first call of
    # each kind is timed on its own: it allocates the stream's workspace and
    # captures the CUDA graphs that later calls replay
    first_call_ms = {}
    for kind, fn in (("lr", lambda: lrcc.lr_rank(succ, head, out=rank_out, stream=stream)),
                     ("cc", lambda: lrcc.cc_label(src, dst, n_cc, out=label, stream=stream))):
        stream.synchronize()
        t0 = time.perf_counter()
        fn()
        stream.synchronize()
        first_call_ms[kind] = (time.perf_counter() - t0) * 1e3
    for _ in range(args.warmup - 1):
        step()
    lrcc.check(stream)
    lr_stats = None

    # timed region: K steps, events on the launching stream, clocks sampled;
    # the library runs as a user would call it (captured CUDA graphs, no
    # instrumentation)
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        stream.synchronize()
    torch.cuda.synchronize()
    barrier()
    clocks = clk.summary()
    ms_step = ev0.elapsed_time(ev1) / args.steps
    lrcc.check(stream)

    # the same steps timed one by one (20 runs, as the paper averages 20):
    # median and minimum
    per_step = []
    for _ in range(20):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        b.synchronize()
        per_step.append(a.elapsed_time(b))
    lrcc.check(stream)
    per_step.sort()
    step_stats = {"runs": len(per_step), "median_ms": (per_step[9] + per_step[10]) / 2, "min_ms": per_step[0],
                  "max_ms": per_step[-1]}

    # the two halves of the step are independent: the same step with the list on
    # one stream and the graph on another (each with its own workspace), joined
    # on the launching stream; K steps, CUDA events on the launching stream
    s_lr, s_cc = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)

    def step_two_streams():
        ev = torch.cuda.Event()
        ev.record(stream)
        s_lr.wait_event(ev)
        s_cc.wait_event(ev)
        lrcc.lr_rank(succ, head, out=rank_out, stream=s_lr)
        lrcc.cc_label(src, dst, n_cc, out=label, stream=s_cc)
        for s_ in (s_lr, s_cc):
            e = torch.cuda.Event()
            e.record(s_)
            stream.wait_event(e)

    for _ in range(args.warmup):
        step_two_streams()
    stream.synchronize()
    t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0e.record(stream)
    for _ in range(args.steps):
        step_two_streams()
    t1e.record(stream)
    stream.synchronize()
    lrcc.check(s_lr)
    lrcc.check(s_cc)
    step_stats["two_streams_ms"] = t0e.elapsed_time(t1e) / args.steps
    step_stats["two_streams_note"] = ("lr_rank and cc_label on two streams of their own, joined each step; the "
                                      "headline value keeps them one after the other on one stream")
    lrcc.release(s_lr)
    lrcc.release(s_cc)

    # second timed pass of K steps with the library's phase timing on: CUDA
    # events on the launching stream around every kernel (plain launches),
    # for the per-kernel durations behind the roofline and the phase split
    lrcc.set_timing(True)
    step()
    stream.synchronize()
    lrcc.phase_times(stream)
    ev2, ev3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev2.record(stream)
    for _ in range(args.steps):
        step()
    ev3.record(stream)
    stream.synchronize()
    ms_step_instrumented = ev2.elapsed_time(ev3) / args.steps
    phases = lrcc.phase_times(stream)
    lrcc.set_timing(False)
    lrcc.check(stream)
    ms_step = max_over_ranks(ms_step)
    value = units * world / (ms_step / 1e3) / 1e6

    # per-part facts
    lrcc.lr_rank(succ, head, out=rank_out, stream=stream)
    lr_stats = lrcc.last_stats(stream)
    lrcc.cc_label(src, dst, n_cc, out=label, stream=stream)
    cc_stats = lrcc.last_stats(stream)
    lrcc.check(stream)

    # the components' ceiling: the hook pass's edge stream and two parent gathers
    # per edge without the hooking (lrcc_gather_probe over the same edges and a
    # table the size of the parent array), timed like the step
    with torch.cuda.stream(stream):
        lrcc.gather_probe(src, dst, label, stream=stream)
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(3):
            lrcc.gather_probe(src, dst, label, stream=stream)
        p1.record(stream)
    stream.synchronize()
    lrcc.check(stream)
    probe_ms = p0.elapsed_time(p1) / 3

    # the first pass over all edges alone: one call with plain launches (the host
    # drives the loop, so each pass is its own launch) and phase timing on
    cc_graphs = lrcc.get_plan(lrcc.KIND_CC, n_cc)["use_graphs"]
    lrcc.set_cc_plan(0, 32, use_graphs=2)
    lrcc.set_timing(True)
    lrcc.cc_label(src, dst, n_cc, out=label, stream=stream)
    lrcc.phase_times(stream)
    full_pass = []
    for _ in range(3):
        lrcc.cc_label(src, dst, n_cc, out=label, stream=stream)
        full_pass.append(lrcc.phase_times(stream).get("cc_hook_full", (float("nan"), 0))[0])
    lrcc.set_timing(False)
    lrcc.set_cc_plan(0, 32, use_graphs=cc_graphs)
    lrcc.check(stream)
    full_pass_ms = min(full_pass)

    lr_ms = sum(v[0] for k, v in phases.items() if k.startswith(("rs_", "lr_small"))) / args.steps
    cc_ms = sum(v[0] for k, v in phases.items() if k.startswith("cc_")) / args.steps
    launches_lr = sum(v[1] for k, v in phases.items() if k.startswith(("rs_", "lr_small")))
    launches_cc = args.steps * (1 + 3 * cc_stats["rounds"])

    hbm, peak_kind = peaks()
    roofline = None
    level0 = lrcc.get_plan(lrcc.KIND_LR, n_lr)["rs_level0"]
    # bytes the method moves: per element of each ruling-set level, per edge read by a hook pass
    lr_method = LR_METHOD_FIRST[level0] * n_lr + 44 * sum(lr_stats["splitters"])
    cc_method = 16 * cc_stats["edges_read"] + 8 * n_cc * cc_stats["rounds"] + 4 * n_cc
    if "rs_walk0" in phases:
        wt, wl = phases["rs_walk0"]
        per_launch_ms = wt / wl
        r1 = lr_stats["splitters"][0] if lr_stats["splitters"] else 0
        if level0 == 2:
            # read succ (4 B) and write the element id (4 B) plus 1 B of chunk header per element;
            # one 8-byte reduced-list word per splitter
            alg_bytes, per_elem = 9 * n_lr + 8 * r1, "9 B per element (read succ, write id + chunk header) + 8 B per splitter"
        else:
            alg_bytes, per_elem = 16 * n_lr + 16 * r1, "16 B per element (read + write back its 8-byte word) + 16 B per splitter"
        achieved = alg_bytes / (per_launch_ms / 1e3) / 1e9
        traffic = None
        if NCU_WALK0["walk_sha1"] == walk0_sha1(os.path.join(ROOT, "paper_1002_4482_gb300", "csrc", "lr.cu")) \
                and args.workload == "large":
            traffic = NCU_WALK0["bytes_per_launch"]
        gather = random_gather_peak(torch, dev, stream)
        chase, chase_chains = chase_peak(lrcc, torch, succ, stream)
        steps_per_s = n_lr / (per_launch_ms / 1e3) / 1e9
        roofline = {"kernel": "rs_walk0c (first-level sublist walk)" if level0 == 2 else "rs_walk (first level)",
                    "bound": "hbm", "achieved": achieved, "peak": hbm, "peak_kind": peak_kind, "unit": "GB/s",
                    "frac": achieved / hbm, "traffic": traffic, "ms_per_launch": per_launch_ms,
                    "algorithmic_bytes": per_elem,
                    "random_access": {
                        "achieved_g_steps_per_s": steps_per_s, "peak_g_per_s": chase,
                        "peak_kind": f"measured here: lrcc_chase_probe, {chase_chains} chains of dependent "
                                     "4-byte reads over the same successor array (the walk's load form, none of "
                                     "its work), best of 2^19 .. 2^23 chains (more than fit at once run in waves)",
                        "frac": steps_per_s / chase,
                        "independent_gathers_g_per_s": gather,
                        "independent_gathers_kind": "torch index_select of 2^28 random 4-byte elements",
                        "frac_of_independent_gathers": steps_per_s / gather,
                        "note": "each walk step is one dependent random read of succ; HBM row activations, "
                                "not bytes, bound random access"}}
        # the other kernels of the step, each against the bound that applies to it
        others = []

        def kernel_row(name, phase, bytes_, note, ceiling=None):
            if phase not in phases:
                return
            ms = phases[phase][0] / phases[phase][1]
            row = {"kernel": name, "ms_per_launch": ms, "algorithmic_bytes": bytes_,
                   "achieved_gbs": bytes_ / (ms / 1e3) / 1e9, "frac_of_hbm": bytes_ / (ms / 1e3) / 1e9 / hbm,
                   "note": note}
            if ceiling:
                row.update(ceiling)
            others.append(row)

        if level0 == 2:
            kernel_row("rs_scatter", "rs_scatter", 13 * n_lr,
                       "5 B read (chunk id + header) + 8 B pair written per element; bound by its shared-memory "
                       "bucket sort")
            kernel_row("rs_place", "rs_expand0", 12 * n_lr,
                       "8 B pair read + 4 B rank written per element; bound by L2 requests (one per random rank "
                       "write)")
        others.append({"kernel": "cc_hook (first pass over all edges)", "ms_per_launch": full_pass_ms,
                       "algorithmic_bytes": 16 * m_cc,
                       "achieved_gbs": 16 * m_cc / (full_pass_ms / 1e3) / 1e9,
                       "frac_of_hbm": 16 * m_cc / (full_pass_ms / 1e3) / 1e9 / hbm,
                       "ceiling_ms": probe_ms, "frac_of_ceiling": probe_ms / full_pass_ms,
                       "note": "8 B edge + two 4-byte parent gathers per edge; ceiling: the gather probe (same "
                               "edge stream and gathers, no hooking), bound by the SM-to-L2 request port"})
        roofline["other_kernels"] = others

    # ordered control and Wyllie baseline on the same list size (not part of the step)
    extra = {}
    if rank == 0:
        def timed(fn, reps=3):
            fn()
            stream.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                fn()
            b.record(stream)
            stream.synchronize()
            return a.elapsed_time(b) / reps
        ms_wy = timed(lambda: lrcc.lr_rank_wyllie(succ, head, out=rank_out, stream=stream), reps=2)
        lrcc.check(stream)
        from gen import workloads
        osucc, ohead = workloads.lr_ordered(28 if args.workload == "large" else 20)
        del succ
        torch.cuda.empty_cache()
        osucc_d = torch.from_numpy(osucc).to(dev)
        ms_ord = timed(lambda: lrcc.lr_rank(osucc_d, ohead, out=rank_out, stream=stream))
        lrcc.check(stream)
        extra = {"lr_wyllie_ms": ms_wy, "lr_wyllie_mnodes_per_s": n_lr / ms_wy / 1e3,
                 "lr_ordered_ms": ms_ord, "lr_ordered_mnodes_per_s": n_lr / ms_ord / 1e3}
        del osucc_d
        succ = torch.from_numpy(succ_h).to(dev)
        # weighted ranks of the same list (values i mod 7, total below 2^31), and of a
        # forest: the same elements cut into 4096 lists (not part of the step)
        with torch.cuda.stream(stream):
            val_d = (torch.arange(n_lr, device=dev, dtype=torch.int64) % 7).to(torch.int32)
        ms_scan = timed(lambda: lrcc.lr_scan(succ, val_d, head, out=rank_out, stream=stream))
        lrcc.check(stream)
        # the forest: the list's order from its ranks, then a tail every n/4096 positions
        lrcc.lr_rank(succ, head, out=rank_out, stream=stream)
        with torch.cuda.stream(stream):
            order = torch.empty(n_lr, dtype=torch.int64, device=dev)
            order[(n_lr - 1 - rank_out).long()] = torch.arange(n_lr, device=dev)
            cuts = torch.linspace(0, n_lr, 4097, device=dev, dtype=torch.float64).long()[1:]
            fsucc = succ.clone()
            fsucc[order[cuts - 1]] = -1
            del order
        ms_forest = timed(lambda: lrcc.lr_scan_forest(fsucc, val_d, out=rank_out, stream=stream), reps=2)
        lrcc.check(stream)
        del fsucc
        extra.update({"lr_scan_ms": ms_scan, "lr_scan_mnodes_per_s": n_lr / ms_scan / 1e3,
                      "lr_scan_forest_ms": ms_forest, "lr_scan_forest_lists": 4096,
                      "lr_scan_forest_mnodes_per_s": n_lr / ms_forest / 1e3})
        del val_d

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        succ_p = torch.from_numpy(succ_h).pin_memory()
        src_p = torch.from_numpy(src_h).pin_memory()
        dst_p = torch.from_numpy(dst_h).pin_memory()
        rank_p = [torch.empty(n_lr, dtype=torch.int32).pin_memory() for _ in range(2)]
        label_p = [torch.empty(n_cc, dtype=torch.int32).pin_memory() for _ in range(2)]
        # consecutive steps alternate between two streams per call, so one step's
        # copies overlap the other's kernels (each stream has its own device staging)
        lr_streams = [torch.cuda.Stream(device=dev) for _ in range(2)]
        cc_streams = [torch.cuda.Stream(device=dev) for _ in range(2)]
        all_streams = lr_streams + cc_streams
        step_no = [0]

        def e2e_step():
            k = step_no[0] % 2
            step_no[0] += 1
            lrcc.lr_rank_host(succ_p, head, out=rank_p[k], stream=lr_streams[k], sync=False)
            lrcc.cc_label_host(src_p, dst_p, n_cc, out=label_p[k], stream=cc_streams[k], sync=False)

        def fork():
            ev = torch.cuda.Event()
            ev.record(stream)
            for s_ in all_streams:
                s_.wait_event(ev)

        def join():
            for s_ in all_streams:
                ev = torch.cuda.Event()
                ev.record(s_)
                stream.wait_event(ev)

        fork()
        for _ in range(args.warmup):
            e2e_step()
        join()
        stream.synchronize()
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fork()
        for _ in range(args.steps):
            e2e_step()
        join()
        b.record(stream)
        stream.synchronize()
        barrier()
        for s_ in all_streams:
            lrcc.check(s_)
        e2e_ms = max_over_ranks(a.elapsed_time(b) / args.steps)
        if rank == 0:
            for k in range(2):
                assert rank_p[k][head].item() == n_lr - 1
                assert int(label_p[k][:4096].max()) <= 4095
        e2e = {"value": units * world / (e2e_ms / 1e3) / 1e6, "unit": UNIT, "ms_per_step": e2e_ms,
               "h2d_bytes_per_step": 4 * n_lr + 8 * m_cc, "d2h_bytes_per_step": 4 * n_lr + 4 * n_cc,
               "api": "lr_rank_host + cc_label_host (host buffers; the library copies in and out)",
               "note": "pinned host buffers; consecutive steps alternate between two streams per call, so one "
                       "step's host-device copies overlap the other step's kernels"}
        # the bound this leg meets: the box's pinned copy rates, measured on the same buffers
        scratch = torch.empty(n_lr, dtype=torch.int32, device=dev)

        def copy_gbs(dst, src):
            with torch.cuda.stream(stream):
                dst.copy_(src, non_blocking=True)
                c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                c0.record(stream)
                for _ in range(3):
                    dst.copy_(src, non_blocking=True)
                c1.record(stream)
            stream.synchronize()
            return 3 * src.numel() * src.element_size() / (c0.elapsed_time(c1) * 1e6)

        h2d_gbs = copy_gbs(scratch, succ_p)
        d2h_gbs = copy_gbs(rank_p[0], scratch)
        del scratch
        bound_ms = max(e2e["h2d_bytes_per_step"] / (h2d_gbs * 1e6), e2e["d2h_bytes_per_step"] / (d2h_gbs * 1e6))
        e2e["copy_bound"] = {"h2d_gbs": h2d_gbs, "d2h_gbs": d2h_gbs, "ms_per_step": bound_ms,
                             "frac": bound_ms / e2e_ms,
                             "note": "pinned 1 GiB copies alone; the step cannot beat its host-to-device bytes at "
                                     "this rate"}
        for s_ in all_streams:
            lrcc.release(s_)
        del succ_p, src_p, dst_p, rank_p, label_p

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample = cpu_sample(args.workload)
        t, tl, tc = time_oracle(sample)
        cpu = {"value": (len(sample[0]) + len(sample[2])) / t / 1e6, "unit": UNIT, "cores": 1,
               "kind": "oracle", "sample": sample[5], "seconds": t, "lr_seconds": tl, "cc_seconds": tc,
               "host_cores": os.cpu_count()}
        # the paper's other CPU comparison: random-splitter list ranking on every host core
        import cpu_baseline
        cores = os.cpu_count() or 1
        cpu_baseline.lr_rank(sample[0], sample[1], cores)
        t0 = time.perf_counter()
        cpu_baseline.lr_rank(sample[0], sample[1], cores)
        tp = time.perf_counter() - t0
        cpu["parallel_lr"] = {"value": len(sample[0]) / tp / 1e6, "unit": "M list nodes/s", "cores": cores,
                              "kind": "random-splitter list ranking, pthreads (cpu_baseline/)",
                              "sample": "the same random-layout list as the oracle leg", "seconds": tp}

    batched = serving = None
    families = sweep = None
    if rank == 0 and not args.no_families:
        families = bench_families(lrcc, torch, dev, stream)
    even = None
    small = None
    if rank == 0 and args.workload == "large":
        small = bench_small_configs(lrcc, torch, dev, stream, hbm)
    if rank == 0 and not args.no_sweep:
        even = bench_even_splitters(lrcc, torch, dev, stream, (16, 20, 24, 28) if args.workload == "large"
                                    else (12, 16, 20))
    if rank == 0 and not args.no_sweep:
        sweep = bench_lr_sweep(lrcc, torch, dev, stream, (16, 18, 20, 22, 24, 26, 28) if args.workload == "large"
                               else (12, 14, 16, 18, 20))
    if not args.no_batched:
        del rank_out, label, src, dst, succ
        torch.cuda.empty_cache()
        barrier()
        batched = bench_batched(lrcc, torch, dev, stream, world=world, rank_id=rank, max_fn=max_over_ranks)
        torch.cuda.empty_cache()
    if rank == 0 and not args.no_serve:
        serving = bench_serve(torch, args.serve_jobs)
        torch.cuda.empty_cache()

    if rank == 0:
        cfg.update({"l2": "inputs larger than L2 (4n B list, 8m B edges); no flush between steps",
                    "parallelism": f"replicas x{world}", "stream": "one non-default stream",
                    "timing": "value: CUDA events on the launching stream around K steps (captured graphs, no "
                              "instrumentation); roofline, lr/cc split and phases: a second pass of K steps with "
                              "CUDA events around every kernel (plain launches)",
                    "ms_per_step_instrumented": ms_step_instrumented})
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "int32", "data": "synthetic (seeded generators in gen/)",
                "config": cfg, "clocks": clocks, "e2e": e2e, "gpu_launches": launches_lr + launches_cc,
                "roofline": roofline, "cpu_baseline": cpu,
                "step_ms": step_stats, "first_call_ms": first_call_ms,
                "lr": {"ms": lr_ms, "mnodes_per_s": n_lr / lr_ms / 1e3 if lr_ms else None,
                       "problem_bytes_frac": 8 * n_lr / (lr_ms / 1e3) / 1e9 / hbm if lr_ms else None,
                       "method_bytes_per_node": lr_method / n_lr,
                       "method_bytes_frac": lr_method / (lr_ms / 1e3) / 1e9 / hbm if lr_ms else None,
                       "method_bytes_note": "first level: " + LR_METHOD_NOTE[level0] + "; each deeper level: "
                                            "8 B read + 8 B written by the select and the walk, 8 B read + "
                                            "4 B written by the expand, per element of the level",
                       "levels": lr_stats["levels"], "splitters": lr_stats["splitters"]},
                "cc": {"ms": cc_ms, "medges_per_s": m_cc / cc_ms / 1e3 if cc_ms else None,
                       "problem_bytes_frac": (8 * m_cc + 4 * n_cc) / (cc_ms / 1e3) / 1e9 / hbm if cc_ms else None,
                       "rounds": cc_stats["rounds"], "edges_read": cc_stats["edges_read"],
                       "method_bytes": cc_method,
                       "method_bytes_frac": cc_method / (cc_ms / 1e3) / 1e9 / hbm if cc_ms else None,
                       "method_bytes_note": "16 B per edge read by a hook pass (8 B of edge, two 4-byte parent "
                                            "gathers), 8 B per vertex and shortcut pass, 4 B per vertex of init; "
                                            "R = rounds",
                       "gather_ceiling": {
                           "probe_ms_per_pass": probe_ms, "probe_gedges_per_s": m_cc / probe_ms / 1e6,
                           "edges_read": cc_stats["edges_read"],
                           "ceiling_ms": cc_stats["edges_read"] / (m_cc / probe_ms),
                           "frac": (cc_stats["edges_read"] / (m_cc / probe_ms)) / cc_ms if cc_ms else None,
                           "full_pass_ms": full_pass_ms, "full_pass_frac": probe_ms / full_pass_ms,
                           "note": "probe: the hook pass's 16-byte edge stream and two gathers per edge (L1, "
                                   "evict-last) over a 4n-byte table, no hooking (lrcc_gather_probe); ceiling: "
                                   "every edge the hook passes read, at the probe's rate; frac = ceiling / cc ms; full_pass: the "
                                   "loop's first pass over all edges alone (plain launches, best of 3), full_pass_frac "
                                   "= probe / full pass"}},
                "phases_ms_per_step": {k: v[0] / args.steps for k, v in phases.items()},
                "batched": batched, "serving": serving, "cc_families": families, "lr_sweep": sweep,
                "even_vs_random_splitters": even, "small_configs": small,
                **extra}
        print(json.dumps(line), flush=True)
    ranks.shutdown()


if __name__ == "__main__":
    main()
