"""Run one call of the library on a seeded input, for profilers (ncu).

    python -m paper_1002_4482_gb300.profile_case lr 26        # lr_rank, random list of 2^26
    python -m paper_1002_4482_gb300.profile_case lr 26 inplace    # or: readonly, split
    python -m paper_1002_4482_gb300.profile_case wyllie 24
    python -m paper_1002_4482_gb300.profile_case cc 22        # cc_label, R-MAT scale 22, edge factor 16
    python -m paper_1002_4482_gb300.profile_case batch 10     # 2^10 mixed instances, both batched calls

Kernels are launched directly (no CUDA-graph replay), so a profiler sees
each of them. The result is checked against the list's closed form, or by
the component invariants, before the script exits 0.
"""
from __future__ import annotations

import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import gen  # noqa: E402
from gen import workloads  # noqa: E402
import paper_1002_4482_gb300 as lrcc  # noqa: E402


def main(argv):
    what, log2 = argv[0], int(argv[1])
    variant = argv[2] if len(argv) > 2 else ""
    dev = torch.device("cuda:0")
    for kind in (lrcc.KIND_LR, lrcc.KIND_LR_WYLLIE, lrcc.KIND_CC, lrcc.KIND_LR_BATCH, lrcc.KIND_CC_BATCH):
        lrcc.set_plan(kind, 0, 32, use_graphs=2)
    if variant == "inplace":
        lrcc.set_plan(lrcc.KIND_LR, 0, 32, rs_level0=1)
    elif variant == "readonly":
        lrcc.set_plan(lrcc.KIND_LR, 0, 32, rs_level0=2)
    elif variant == "split":
        lrcc.set_plan(lrcc.KIND_LR, 0, 32, rs_level0=3)
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
        lab = lrcc.cc_label(torch.from_numpy(src).to(dev), torch.from_numpy(dst).to(dev), n)
        lrcc.check()
        lab = lab.cpu().numpy()
        assert np.array_equal(lab[src], lab[dst]) and (lab <= np.arange(n)).all()
        print("rounds", lrcc.last_stats()["rounds"])
    elif what == "batch":
        (succ, off, heads), (src, dst, eoff, voff) = workloads.batch(1 << log2)
        lrcc.lr_rank_batched(*(torch.from_numpy(x).to(dev) for x in (succ, off, heads)))
        lrcc.cc_label_batched(*(torch.from_numpy(x).to(dev) for x in (src, dst, eoff, voff)))
        lrcc.check()
    else:
        raise SystemExit(f"unknown case {what}")
    torch.cuda.synchronize()
    print("ok", what, log2, variant)


if __name__ == "__main__":
    main(sys.argv[1:])
