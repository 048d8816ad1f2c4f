"""Weighted list ranking (lr_scan, lr_scan_forest): the CUDA path against the
oracle, element by element, bit-exact (sums modulo 2^32)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1002_4482_gb300 as lrcc

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.int32)).to(DEV)


def _scan(succ, val, head):
    out = lrcc.lr_scan(_dev(succ), _dev(val), head)
    lrcc.check()
    return out.cpu().numpy()


def _forest(succ, val):
    out = lrcc.lr_scan_forest(_dev(succ), _dev(val))
    lrcc.check()
    return out.cpu().numpy()


@pytest.mark.parametrize("n", [1, 2, 5, 4096, 8193, 16385, 100_003, 1 << 20])
@pytest.mark.parametrize("seed", [1, 2])
def test_scan_matches_oracle(n, seed):
    succ, head = gen.list_random(n, 70 + seed)
    val = np.random.default_rng(n + seed).integers(0, 1000, n).astype(np.int32)
    assert np.array_equal(_scan(succ, val, head), oracle.lr_scan(succ, val, head))


def test_scan_unit_values_is_rank_plus_one():
    succ, head = gen.list_random(300_007, 73)
    ones = np.ones(len(succ), np.int32)
    rank = lrcc.lr_rank(_dev(succ), head).cpu().numpy()
    assert np.array_equal(_scan(succ, ones, head), rank + 1)


def test_scan_large_values_and_ordered_layout():
    # totals up to 2^31 - 1, the top of the supported range
    for n, (succ, head) in ((200_000, gen.list_random(200_000, 74)), (200_000, gen.list_ordered(200_000)),
                            (5000, gen.list_random(5000, 75))):
        val = np.full(n, (2**31 - 1) // n, np.int32)
        val[0] += (2**31 - 1) - int(val.astype(np.int64).sum())
        assert int(val.astype(np.int64).sum()) == 2**31 - 1
        assert np.array_equal(_scan(succ, val, head), oracle.lr_scan(succ, val, head))


@pytest.mark.parametrize("n", [5000, 300_000])
@pytest.mark.parametrize("case", ["negative", "total_too_large"])
def test_scan_values_out_of_range_are_reported(n, case):
    succ, head = gen.list_random(n, 80)
    val = np.ones(n, np.int32)
    if case == "negative":
        val[n // 2] = -1
    else:
        val[:] = (2**31) // n + 1
    lrcc.lr_scan(_dev(succ), _dev(val), head)
    assert lrcc.last_status() == lrcc.ERR_INVALID_INPUT
    # the next valid call is unaffected
    ok = np.ones(n, np.int32)
    assert np.array_equal(_scan(succ, ok, head), oracle.lr_scan(succ, ok, head))


def test_scan_under_every_first_level_plan():
    # the scan always takes the in-place first level, whatever the table says
    succ, head = gen.list_random(400_000, 75)
    val = np.random.default_rng(5).integers(0, 50, len(succ)).astype(np.int32)
    expect = oracle.lr_scan(succ, val, head)
    try:
        for l0, d0 in ((1, 8), (2, 32), (1, 256), (2, 4)):
            lrcc.set_plan(lrcc.KIND_LR, 0, 32, rs_level0=l0, rs_spacing0=d0)
            assert np.array_equal(_scan(succ, val, head), expect), (l0, d0)
    finally:
        lrcc.reset_plans()


@pytest.mark.parametrize("n", [7, 20_000, 300_000])
@pytest.mark.parametrize("case", ["cycle", "two_lists", "out_of_range"])
def test_scan_invalid_inputs_are_reported(n, case):
    succ, head = gen.list_random(n, 76)
    succ = succ.copy()
    tail = int(np.flatnonzero(succ == -1)[0])
    if case == "cycle":
        succ[tail] = head
    elif case == "two_lists":
        # cut the list in two after its head's successor
        succ[succ[head]] = -1
    else:
        succ[tail] = n + 5
    lrcc.lr_scan(_dev(succ), _dev(np.ones(n, np.int32)), head)
    assert lrcc.last_status() == lrcc.ERR_INVALID_INPUT


@pytest.mark.parametrize("sizes", [[1], [3, 1, 4, 1, 5], [100_000], [2] * 5000, [70_000, 1, 30_000, 999, 12]])
def test_forest_matches_oracle(sizes):
    n = sum(sizes)
    perm = gen.permutation(n, 77)
    succ = np.full(n, -1, np.int32)
    at = 0
    for k, sz in enumerate(sizes):
        piece = perm[at:at + sz]
        succ[piece[:-1]] = piece[1:]
        if k % 2:
            succ[piece[-1]] = piece[-1]            # the paper's self-loop tail
        at += sz
    val = np.random.default_rng(n).integers(-100, 100, n).astype(np.int32)
    assert np.array_equal(_forest(succ, val), oracle.lr_scan_forest(succ, val))


def test_forest_of_one_list_equals_scan():
    succ, head = gen.list_random(250_000, 78)
    val = np.random.default_rng(8).integers(0, 9, len(succ)).astype(np.int32)
    assert np.array_equal(_forest(succ, val), _scan(succ, val, head))


def test_forest_sums_wrap_modulo_2_32():
    # the forest form has no range limit: negative values and wrapping sums
    n = 100_000
    succ, head = gen.list_random(n, 81)
    val = np.full(n, 2**31 - 3, np.int32)
    val[::7] = -(2**31)
    assert np.array_equal(_forest(succ, val), oracle.lr_scan_forest(succ, val))


def test_forest_large_totals_take_the_pointer_jumping_form():
    # non-negative values whose total passes 2^31: the first level's 31-bit fields cannot
    # hold the sums, so the whole forest is summed by pointer jumping (no error)
    n = 300_000
    perm = gen.permutation(n, 82)
    succ = np.full(n, -1, np.int32)
    for piece in np.array_split(perm, 7):
        succ[piece[:-1]] = piece[1:]
    val = np.full(n, 2**31 // n + 100, np.int32)
    assert np.array_equal(_forest(succ, val), oracle.lr_scan_forest(succ, val))


@pytest.mark.parametrize("case", ["named_twice", "cycle", "out_of_range"])
def test_forest_invalid_inputs_are_reported(case):
    n = 10_000
    succ, head = gen.list_random(n, 79)
    succ = succ.copy()
    tail = int(np.flatnonzero(succ == -1)[0])
    if case == "named_twice":
        succ[tail] = succ[head]                    # two predecessors of one element
    elif case == "cycle":
        succ[tail] = head
    else:
        succ[tail] = -7
    lrcc.lr_scan_forest(_dev(succ), _dev(np.ones(n, np.int32)))
    assert lrcc.last_status() == lrcc.ERR_INVALID_INPUT


@pytest.mark.slow
def test_scan_full_size_2p28():
    # closed form over the generator's layout: out[perm[k]] = sum of val[perm[j]], j >= k (uint32)
    n = 1 << 28
    succ, head, perm = gen.list_random(n, 3, with_perm=True)
    val = (np.arange(n, dtype=np.int64) % 7).astype(np.int32)   # total 805306362 < 2^31
    out = lrcc.lr_scan(_dev(succ), _dev(val), head)
    lrcc.check()
    v = val[perm].astype(np.uint32)
    suf = np.cumsum(v[::-1], dtype=np.uint32)[::-1].view(np.int32)
    assert np.array_equal(out.cpu().numpy()[perm], suf)
