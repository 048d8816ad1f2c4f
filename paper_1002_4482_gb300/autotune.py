"""Autotuner for the library's plan table.

For each size class it times candidate plans on seeded synthetic inputs of
that size and installs the fastest one with ``set_plan`` for the size range
the class stands for. Every candidate's output is checked before its time
counts, so a wrong plan can never win:

  lists       ranks against the generator's closed form: the generator returns
              the permutation it laid each list out by, and the element at
              position k of a list of n elements has rank n - 1 - k;
  graphs      labels equal, element by element, to those of the reference plan
              (hook rule 1, no sample pass, plain launches: the simplest form of
              the method, the one the parity tests pin), computed once per input
              on the GPU before any candidate runs. Min-id labels are unique, so
              a candidate that merges or splits a component differs there.

Knobs searched:
  lists       first-level mode (in-place words / read-only walk), spacing at the
              first and deeper levels, walks per thread, one-block cutoff
  components  hook rule (single hook / re-link / single then re-link), sample pass size, for
              graphs with at least 4 edges per vertex and, apart, for sparser ones
  batched     minimum splitter spacing of in-block ruling sets; hook rule of the
              large-graph union path

Results are cached as JSON keyed by GPU name, so ``load`` can apply them in
later processes without tuning again::

    python -m paper_1002_4482_gb300.autotune --out plans.json [--quick]
"""
from __future__ import annotations

import argparse
import itertools
import json
import os
import sys
import time

import numpy as np
import torch

from . import (KIND_CC, KIND_CC_BATCH, KIND_CC_SPARSE, KIND_LR, KIND_LR_BATCH, cc_label, cc_label_batched, check,
               get_plan, lr_rank, lr_rank_batched, set_plan)


def _timeit(fn, stream, reps=3):
    fn()
    stream.synchronize()
    check(stream)
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    check(stream)
    return best


def _lr_candidates(log2n, quick):
    # first-level layouts: in-place words, read-only walk (from 2^22), and in the
    # full search the split mark / rank arrays as well
    level0 = ((1, 2) if log2n >= 22 else (1,)) + (() if quick else (3,))
    sp0 = (8, 32) if quick else (8, 16, 32, 64)
    sp = (8,) if quick else (4, 8, 16, 32)
    small = (16384,) if quick else (4096, 8192, 16384)
    chains = (1,) if quick else (1, 2)
    for l0, d0, d, sm, ch in itertools.product(level0, sp0, sp, small, chains):
        yield {"rs_level0": l0, "rs_spacing0": d0, "rs_spacing": d, "rs_small": sm, "rs_chains": ch}


def _ranges(classes):
    """Size range [lo, hi] of ceil(log2 n) that each tuned class stands for."""
    out, cs = [], sorted(classes)
    for i, c in enumerate(cs):
        lo = 0 if i == 0 else (cs[i - 1] + c) // 2 + 1
        hi = 32 if i == len(cs) - 1 else (c + cs[i + 1]) // 2
        out.append((c, lo, hi))
    return out


def tune_lists(classes=(16, 20, 24, 28), quick=False, device=0, log=print):
    import gen
    dev = torch.device("cuda", device)
    stream = torch.cuda.Stream(dev)
    results = {}
    for c, lo, hi in _ranges(classes):
        n = 1 << c
        succ, head, perm = gen.list_random(n, 100 + c, with_perm=True)
        with torch.cuda.stream(stream):
            s = torch.from_numpy(succ).to(dev)
            out = torch.empty_like(s)
            perm_d = torch.from_numpy(perm).to(dev).long()
            expect = torch.arange(n - 1, -1, -1, dtype=torch.int32, device=dev)
        best = None
        for cand in _lr_candidates(c, quick or c >= 26):
            set_plan(KIND_LR, c, c, **cand)
            ms = _timeit(lambda: lr_rank(s, head, out=out, stream=stream), stream)
            with torch.cuda.stream(stream):
                ok = bool(torch.equal(out[perm_d], expect))
            if not ok:
                raise AssertionError(f"plan {cand} gave wrong ranks at n = 2^{c}")
            if best is None or ms < best[0]:
                best = (ms, cand)
        set_plan(KIND_LR, lo, hi, **best[1])
        results[str(c)] = {"range": [lo, hi], "ms": best[0], "plan": best[1]}
        log(f"lists 2^{c}: {best[0]:.3f} ms with {best[1]}")
        del s, out, perm_d, expect
    return results


# Plan the tuner takes the expected component labels from.
REFERENCE_CC = {"cc_hook": 1, "cc_sample": 1, "use_graphs": 2}


def _reference_labels(kind, log2_lo, log2_hi, run):
    """Labels of `run()` under the reference plan, with the plan table restored after."""
    saved = get_plan(kind, 1 << log2_lo)
    set_plan(kind, log2_lo, log2_hi, **REFERENCE_CC)
    try:
        return run().clone()
    finally:
        set_plan(kind, log2_lo, log2_hi, **{k: saved[k] for k in ("cc_hook", "cc_sample", "use_graphs")})


def tune_graphs(classes=(16, 20, 24), device=0, log=print, sparse=False):
    """Hook rule and sample pass per size class. Dense (KIND_CC): R-MAT graphs
    of 16 edges per vertex and uniform random graphs of 4; sparse
    (KIND_CC_SPARSE, fewer than 4 edges per vertex): uniform random graphs of 2
    and collections of paths."""
    import gen
    from gen import workloads
    dev = torch.device("cuda", device)
    stream = torch.cuda.Stream(dev)
    kind = KIND_CC_SPARSE if sparse else KIND_CC
    results = {}
    for c, lo, hi in _ranges(classes):
        if sparse:
            src1, dst1 = gen.er(1 << c, 1 << (c + 1), 400 + c)
            n1 = 1 << c
            src2, dst2, n2 = gen.list_graph(16, (1 << c) // 16, 500 + c)
        else:
            # a mix of the two graph families the library is measured on
            src1, dst1, n1 = workloads.cc_rmat(c, 16, seed=200 + c)
            src2, dst2 = gen.er(1 << c, 1 << (c + 2), 300 + c)
            n2 = 1 << c
        cases = []
        with torch.cuda.stream(stream):
            for s_, d_, n_ in ((src1, dst1, n1), (src2, dst2, n2)):
                cases.append((torch.from_numpy(s_).to(dev), torch.from_numpy(d_).to(dev), n_,
                              torch.empty(n_, dtype=torch.int32, device=dev), s_, d_))
        expect = []
        for sd, dd, n_, lab, _, _ in cases:
            def run(sd=sd, dd=dd, n_=n_, lab=lab):
                cc_label(sd, dd, n_, out=lab, stream=stream)
                stream.synchronize()
                check(stream)
                return lab
            expect.append(_reference_labels(kind, c, c, run))
        best = None
        for hook, samp in itertools.product((1, 2, 3, 5), (-1, 1, 4, 8)):
            set_plan(kind, c, c, cc_hook=hook, cc_sample=samp, use_graphs=1)
            ms = 0.0
            for (sd, dd, n_, lab, _, _), want in zip(cases, expect):
                ms += _timeit(lambda: cc_label(sd, dd, n_, out=lab, stream=stream), stream)
                with torch.cuda.stream(stream):
                    ok = bool(torch.equal(lab, want))
                if not ok:
                    raise AssertionError(f"hook rule {hook}, sample {samp} gave labels unlike the reference "
                                         f"plan's at 2^{c}")
            if best is None or ms < best[0]:
                best = (ms, {"cc_hook": hook, "cc_sample": samp})
        set_plan(kind, lo, hi, **best[1])
        results[str(c)] = {"range": [lo, hi], "ms": best[0], "plan": best[1]}
        log(f"{'sparse ' if sparse else ''}graphs 2^{c}: {best[0]:.3f} ms with {best[1]}")
    return results


def _batch_expected_ranks(off: np.ndarray, perm: np.ndarray) -> np.ndarray:
    """Closed form of batched random lists: the element at position j of list k
    (local id perm[off[k] + j]) has rank size_k - 1 - j."""
    total = int(off[-1])
    sizes = np.diff(off)
    start = np.repeat(off[:-1], sizes)
    end = np.repeat(off[1:], sizes)
    want = np.empty(total, np.int32)
    want[start + perm] = (end - 1 - np.arange(total, dtype=np.int64)).astype(np.int32)
    return want


def tune_batched(log2_count=10, device=0, log=print):
    from gen import workloads
    dev = torch.device("cuda", device)
    stream = torch.cuda.Stream(dev)
    (succ, off, heads, perm), (src, dst, eoff, voff) = workloads.batch(1 << log2_count, with_perm=True)
    with torch.cuda.stream(stream):
        S, O, H = (torch.from_numpy(x).to(dev) for x in (succ, off, heads))
        SR, DS, EO, VO = (torch.from_numpy(x).to(dev) for x in (src, dst, eoff, voff))
        rank = torch.empty_like(S)
        lab = torch.empty(int(voff[-1]), dtype=torch.int32, device=dev)
    want_r = _batch_expected_ranks(off, perm)

    def run_graphs():
        cc_label_batched(SR, DS, EO, VO, n_total=int(voff[-1]), out=lab, stream=stream)
        stream.synchronize()
        check(stream)
        return lab
    want_l = _reference_labels(KIND_CC_BATCH, 0, 32, run_graphs).cpu().numpy()
    res = {}
    best = None
    for d in (4, 16, 64):
        set_plan(KIND_LR_BATCH, 0, 32, rs_spacing0=d)
        ms = _timeit(lambda: lr_rank_batched(S, O, H, out=rank, stream=stream), stream)
        if not np.array_equal(rank.cpu().numpy(), want_r):
            raise AssertionError(f"batched spacing {d} gave wrong ranks")
        if best is None or ms < best[0]:
            best = (ms, {"rs_spacing0": d})
    set_plan(KIND_LR_BATCH, 0, 32, **best[1])
    res["lists"] = {"ms": best[0], "plan": best[1]}
    log(f"batched lists: {best[0]:.3f} ms with {best[1]}")
    best = None
    for hook in (1, 2, 5):
        set_plan(KIND_CC_BATCH, 0, 32, cc_hook=hook)
        ms = _timeit(lambda: cc_label_batched(SR, DS, EO, VO, n_total=int(voff[-1]), out=lab, stream=stream), stream)
        if not np.array_equal(lab.cpu().numpy(), want_l):
            raise AssertionError(f"batched hook rule {hook} gave wrong labels")
        if best is None or ms < best[0]:
            best = (ms, {"cc_hook": hook})
    set_plan(KIND_CC_BATCH, 0, 32, **best[1])
    res["graphs"] = {"ms": best[0], "plan": best[1]}
    log(f"batched graphs: {best[0]:.3f} ms with {best[1]}")
    return res


def tune(quick=False, device=0, log=print, list_classes=(16, 20, 24, 28), graph_classes=(16, 20, 24),
         batch_log2=10) -> dict:
    t0 = time.time()
    out = {"gpu": torch.cuda.get_device_name(device), "quick": quick,
           "lists": tune_lists(list_classes, quick, device, log),
           "graphs": tune_graphs(graph_classes, device, log),
           "sparse_graphs": tune_graphs(graph_classes, device, log, sparse=True),
           "batched": tune_batched(batch_log2, device, log)}
    out["seconds"] = time.time() - t0
    return out


def apply(result: dict) -> None:
    """Install a tuning result (as returned by tune or read from a cache)."""
    for entry in result.get("lists", {}).values():
        set_plan(KIND_LR, entry["range"][0], entry["range"][1], **entry["plan"])
    for entry in result.get("graphs", {}).values():
        set_plan(KIND_CC, entry["range"][0], entry["range"][1], **entry["plan"])
    for entry in result.get("sparse_graphs", {}).values():
        set_plan(KIND_CC_SPARSE, entry["range"][0], entry["range"][1], **entry["plan"])
    b = result.get("batched", {})
    if "lists" in b:
        set_plan(KIND_LR_BATCH, 0, 32, **b["lists"]["plan"])
    if "graphs" in b:
        set_plan(KIND_CC_BATCH, 0, 32, **b["graphs"]["plan"])


def load(path: str, device: int = 0) -> bool:
    """Apply a cached result if it was tuned on the same kind of GPU."""
    if not os.path.exists(path):
        return False
    with open(path) as f:
        result = json.load(f)
    if result.get("gpu") != torch.cuda.get_device_name(device):
        return False
    apply(result)
    return True


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--out", default="lrcc_plans.json")
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--device", type=int, default=0)
    args = ap.parse_args(argv)
    res = tune(args.quick, args.device)
    with open(args.out, "w") as f:
        json.dump(res, f, indent=1)
    print(json.dumps({"out": args.out, "seconds": res["seconds"]}))


if __name__ == "__main__":
    sys.exit(main())
