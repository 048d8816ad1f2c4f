"""Batched list ranking and components: every instance of a batch must equal
the oracle on that instance alone (bit-exact)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1002_4482_gb300 as lrcc
from gen import workloads

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _lists(sizes, seed):
    succ, off, heads = gen.list_batch(np.asarray(sizes, np.int64), seed)
    rank = lrcc.lr_rank_batched(torch.from_numpy(succ).to(DEV), torch.from_numpy(off).to(DEV),
                                torch.from_numpy(heads).to(DEV))
    lrcc.check()
    return succ, off, heads, rank.cpu().numpy()


def _graphs(vsizes, seed, deg=2):
    src, dst, eoff, voff = gen.er_batch(np.asarray(vsizes, np.int64), deg, 1, seed)
    lab = lrcc.cc_label_batched(torch.from_numpy(src).to(DEV), torch.from_numpy(dst).to(DEV),
                                torch.from_numpy(eoff).to(DEV), torch.from_numpy(voff).to(DEV))
    lrcc.check()
    return src, dst, eoff, voff, lab.cpu().numpy()


@pytest.mark.parametrize("seed", [1, 2])
def test_list_batch_mixed_sizes(seed):
    # one-block path (<= 8192), in-block ruling set (> 8192), tiny and ragged sizes
    sizes = [1, 2, 3, 31, 33, 1000, 8191, 8192, 8193, 9000, 20000, 65537, 300000] + \
        gen.loguniform_sizes(60, 0, 17, seed).tolist()
    succ, off, heads, rank = _lists(sizes, seed)
    assert np.array_equal(rank, oracle.lr_rank_batched(succ, off, heads))


@pytest.mark.parametrize("seed", [1, 2])
def test_graph_batch_mixed_sizes(seed):
    # shared-memory path (<= 16384 vertices) and global path, degree 4 and 0.5
    sizes = [1, 2, 5, 100, 16383, 16384, 16385, 50000, 200000] + gen.loguniform_sizes(60, 0, 17, seed).tolist()
    for deg in (2, 1):
        src, dst, eoff, voff, lab = _graphs(sizes, seed, deg)
        assert np.array_equal(lab, oracle.cc_batched(src, dst, eoff, voff))


@pytest.mark.parametrize("hook", [1, 5])
def test_graph_batch_of_consecutive_id_paths(hook):
    # paths whose edges join consecutive local ids, in id order: a deep chain per
    # instance after the first hook pass, in the shared-memory path (<= 2^15
    # vertices) and in the union of the large instances; every label is 0
    sizes = [2, 1000, 1 << 15, (1 << 15) + 1, 1 << 17, 300_000]
    src = np.concatenate([np.arange(k - 1, dtype=np.int32) for k in sizes])
    dst = np.concatenate([np.arange(1, k, dtype=np.int32) for k in sizes])
    eoff = np.concatenate([[0], np.cumsum([k - 1 for k in sizes])]).astype(np.int64)
    voff = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    lrcc.set_plan(lrcc.KIND_CC_BATCH, 0, 32, cc_hook=hook)
    try:
        lab = lrcc.cc_label_batched(*(torch.from_numpy(x).to(DEV) for x in (src, dst, eoff, voff)))
        lrcc.check()
    finally:
        lrcc.reset_plans()
    assert not lab.any().item()


def test_batch_with_empty_instances():
    sizes = [0, 5, 0, 0, 10000, 0]
    succ, off, heads, rank = _lists(sizes, 3)
    expect = oracle.lr_rank_batched(succ, off, heads)
    assert np.array_equal(rank, expect)
    src, dst, eoff, voff, lab = _graphs([0, 3, 0, 20000], 4)
    assert np.array_equal(lab, oracle.cc_batched(src, dst, eoff, voff))


def test_batch_result_equals_single_calls():
    sizes = gen.loguniform_sizes(24, 8, 16, 9)
    succ, off, heads, rank = _lists(sizes, 9)
    for k in range(len(sizes)):
        b, e = off[k], off[k + 1]
        single = lrcc.lr_rank(torch.from_numpy(succ[b:e].copy()).to(DEV), int(heads[k])).cpu().numpy()
        assert np.array_equal(rank[b:e], single)
    src, dst, eoff, voff, lab = _graphs(sizes, 10)
    for k in range(len(sizes)):
        eb, ee, vb, ve = eoff[k], eoff[k + 1], voff[k], voff[k + 1]
        single = lrcc.cc_label(torch.from_numpy(src[eb:ee].copy()).to(DEV),
                               torch.from_numpy(dst[eb:ee].copy()).to(DEV), int(ve - vb)).cpu().numpy()
        assert np.array_equal(lab[vb:ve], single)


def test_invalid_instance_is_reported():
    sizes = [100, 20000, 50]
    succ, off, heads = gen.list_batch(np.asarray(sizes, np.int64), 5)
    succ = succ.copy()
    b = off[1]
    tail = b + int(np.flatnonzero(succ[b:off[2]] == -1)[0])
    succ[tail] = heads[1]                      # list 1 becomes a cycle
    lrcc.lr_rank_batched(torch.from_numpy(succ).to(DEV), torch.from_numpy(off).to(DEV),
                         torch.from_numpy(heads).to(DEV))
    assert lrcc.last_status() == lrcc.ERR_INVALID_INPUT
    heads2 = heads.copy()
    heads2[2] = 50                             # head outside its list
    succ, off, _ = gen.list_batch(np.asarray(sizes, np.int64), 5)
    lrcc.lr_rank_batched(torch.from_numpy(succ).to(DEV), torch.from_numpy(off).to(DEV),
                         torch.from_numpy(heads2).to(DEV))
    assert lrcc.last_status() == lrcc.ERR_INVALID_INPUT
    src, dst, eoff, voff = gen.er_batch(np.asarray([10, 10], np.int64), 2, 1, 6)
    dst = dst.copy()
    dst[25] = 10                               # endpoint outside graph 1
    lrcc.cc_label_batched(torch.from_numpy(src).to(DEV), torch.from_numpy(dst).to(DEV),
                          torch.from_numpy(eoff).to(DEV), torch.from_numpy(voff).to(DEV))
    assert lrcc.last_status() == lrcc.ERR_INVALID_INPUT


def test_plain_entry_point_reads_total_itself():
    # lr_rank_batched (not _sized) takes the total from node_off on the device
    import ctypes
    sizes = [7, 9000, 3]
    succ, off, heads = gen.list_batch(np.asarray(sizes, np.int64), 8)
    s, o, h = (torch.from_numpy(x).to(DEV) for x in (succ, off, heads))
    rank = torch.empty_like(s)
    st = lrcc.load().lr_rank_batched(s.data_ptr(), o.data_ptr(), h.data_ptr(), len(sizes), rank.data_ptr(),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == lrcc.OK
    lrcc.check()
    assert np.array_equal(rank.cpu().numpy(), oracle.lr_rank_batched(succ, off, heads))


@pytest.mark.slow
def test_full_size_4096_batch():
    # the batched workload: 2048 lists + 2048 graphs of degree 4, sizes log-uniform in [2^8, 2^20)
    (succ, off, heads), (src, dst, eoff, voff) = workloads.batch(4096)
    rank = lrcc.lr_rank_batched(torch.from_numpy(succ).to(DEV), torch.from_numpy(off).to(DEV),
                                torch.from_numpy(heads).to(DEV))
    lab = lrcc.cc_label_batched(torch.from_numpy(src).to(DEV), torch.from_numpy(dst).to(DEV),
                                torch.from_numpy(eoff).to(DEV), torch.from_numpy(voff).to(DEV))
    lrcc.check()
    assert np.array_equal(rank.cpu().numpy(), oracle.lr_rank_batched(succ, off, heads))
    assert np.array_equal(lab.cpu().numpy(), oracle.cc_batched(src, dst, eoff, voff))


def test_plain_graph_entry_point_reads_total_itself():
    import ctypes
    src, dst, eoff, voff = gen.er_batch(np.asarray([100, 40000, 70000, 3], np.int64), 2, 1, 12)
    a, b, eo, vo = (torch.from_numpy(x).to(DEV) for x in (src, dst, eoff, voff))
    lab = torch.empty(int(voff[-1]), dtype=torch.int32, device=DEV)
    st = lrcc.load().cc_label_batched(a.data_ptr(), b.data_ptr(), eo.data_ptr(), vo.data_ptr(), 4, lab.data_ptr(),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == lrcc.OK
    lrcc.check()
    assert np.array_equal(lab.cpu().numpy(), oracle.cc_batched(src, dst, eoff, voff))


@pytest.mark.parametrize("seed", [1, 2])
def test_large_batches_ranked_as_one_list(seed):
    # at least 2^25 elements in all (where the built-in plan takes the read-only first
    # level): the lists are linked into one list; empty lists, one-element lists,
    # self-loop tails
    sizes = [0, 1, 2, 5, 1000, 1 << 20, 0, 0, 3, (1 << 24) + 7, 77_777, 1] + \
        gen.loguniform_sizes(300, 0, 16, seed).tolist() + [(1 << 24) + 1000]
    assert sum(sizes) >= 1 << 25
    succ, off, heads = gen.list_batch(np.asarray(sizes, np.int64), 30 + seed)
    succ = succ.copy()
    for k in range(0, len(sizes), 3):                   # every third list ends in a self-loop
        b, e = off[k], off[k + 1]
        if e > b:
            tail = b + int(np.flatnonzero(succ[b:e] == -1)[0])
            succ[tail] = tail - b
    rank = lrcc.lr_rank_batched(torch.from_numpy(succ).to(DEV), torch.from_numpy(off).to(DEV),
                                torch.from_numpy(heads).to(DEV))
    lrcc.check()
    assert np.array_equal(rank.cpu().numpy(), oracle.lr_rank_batched(succ, off, heads))


@pytest.mark.parametrize("case", ["cycle", "two_lists", "head_out_of_range", "succ_out_of_range"])
def test_large_batch_invalid_instance_is_reported(case):
    sizes = [100, 1 << 24, 50, (1 << 24) + 3]
    succ, off, heads = gen.list_batch(np.asarray(sizes, np.int64), 40)
    succ, heads = succ.copy(), heads.copy()
    b, e = off[1], off[2]
    tail = b + int(np.flatnonzero(succ[b:e] == -1)[0])
    if case == "cycle":
        succ[tail] = heads[1]
    elif case == "two_lists":
        succ[b + heads[1]] = -1
    elif case == "head_out_of_range":
        heads[3] = sizes[3]
    else:
        succ[tail] = sizes[1]
    lrcc.lr_rank_batched(torch.from_numpy(succ).to(DEV), torch.from_numpy(off).to(DEV),
                         torch.from_numpy(heads).to(DEV))
    assert lrcc.last_status() == lrcc.ERR_INVALID_INPUT


def test_large_batch_with_the_in_place_plan_takes_the_block_path():
    # rs_level0 = 1 in the batched plan keeps every list on the per-block kernel
    sizes = [1 << 24, 3, (1 << 24) + 1, 0, 999]
    succ, off, heads = gen.list_batch(np.asarray(sizes, np.int64), 41)
    lrcc.set_plan(lrcc.KIND_LR_BATCH, 0, 32, rs_level0=1)
    try:
        rank = lrcc.lr_rank_batched(torch.from_numpy(succ).to(DEV), torch.from_numpy(off).to(DEV),
                                    torch.from_numpy(heads).to(DEV))
        lrcc.check()
    finally:
        lrcc.reset_plans()
    assert np.array_equal(rank.cpu().numpy(), oracle.lr_rank_batched(succ, off, heads))


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_shares_gather_to_the_whole_batch(world):
    # the batched calls on each rank's LPT share (run here one share after the
    # other on one GPU), put back in place: equal to the oracle on the whole batch
    from paper_1002_4482_gb300 import shard
    (succ, off, heads), (src, dst, eoff, voff) = workloads.batch(256, 6.0, 17.0, seed=21)
    rank_all = np.full(len(succ), -9, np.int32)
    lab_all = np.full(int(voff[-1]), -9, np.int32)
    for idx in shard.lpt_assign(shard.list_costs(off), world):
        s, o, h = shard.list_share(succ, off, heads, idx)
        r = lrcc.lr_rank_batched(*(torch.from_numpy(x).to(DEV) for x in (s, o, h)))
        lrcc.check()
        shard.scatter_back(rank_all, off, idx, r.cpu().numpy())
    for idx in shard.lpt_assign(shard.graph_costs(eoff, voff), world):
        a, b, eo, vo = shard.graph_share(src, dst, eoff, voff, idx)
        lab = lrcc.cc_label_batched(*(torch.from_numpy(x).to(DEV) for x in (a, b, eo, vo)))
        lrcc.check()
        shard.scatter_back(lab_all, voff, idx, lab.cpu().numpy())
    assert np.array_equal(rank_all, oracle.lr_rank_batched(succ, off, heads))
    assert np.array_equal(lab_all, oracle.cc_batched(src, dst, eoff, voff))
