"""lr_rank_noalloc, the list-ranking entry point for callers that cannot
allocate device memory (its scratch is a fixed device array inside the
library), must give exactly the ranks of lr_rank. Called through the C ABI."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import gen
import paper_1002_4482_gb300 as lrcc

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _noalloc(succ: torch.Tensor, head: int, out: torch.Tensor) -> int:
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lrcc.load().lr_rank_noalloc(ctypes.c_void_p(succ.data_ptr()), succ.numel(), int(head),
                                       ctypes.c_void_p(out.data_ptr()), stream)


def test_noalloc_matches_lr_rank_on_two_calls_in_a_row():
    # the largest size first, then a smaller one: the shared scratch still
    # holds the first call's contents when the second call starts
    for n, seed in ((1 << 20, 11), (300_001, 12)):
        succ, head = gen.list_random(n, seed)
        s = torch.from_numpy(succ).to(DEV)
        expect = lrcc.lr_rank(s, head)
        lrcc.check()
        out = torch.full_like(s, -7)
        assert _noalloc(s, head, out) == lrcc.OK
        torch.cuda.synchronize()
        assert torch.equal(out, expect)


def test_noalloc_one_block_size_and_limits():
    succ, head = gen.list_random(5000, 13)
    s = torch.from_numpy(succ).to(DEV)
    out = torch.empty_like(s)
    assert _noalloc(s, head, out) == lrcc.OK
    torch.cuda.synchronize()
    assert torch.equal(out, lrcc.lr_rank(s, head))
    big = torch.zeros((1 << 20) + 1, dtype=torch.int32, device=DEV)
    assert _noalloc(big, 0, torch.empty_like(big)) == lrcc.ERR_ARG


def test_noalloc_reports_invalid_input_in_the_output():
    succ, head = gen.list_random(100_000, 14)
    succ = succ.copy()
    succ[int(np.flatnonzero(succ == -1)[0])] = head      # the list becomes a cycle
    s = torch.from_numpy(succ).to(DEV)
    out = torch.empty_like(s)
    assert _noalloc(s, head, out) == lrcc.OK
    torch.cuda.synchronize()
    assert out[head].item() == -1
