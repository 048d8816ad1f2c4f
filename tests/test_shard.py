"""Batched instances sharded over ranks (paper_1002_4482_gb300.shard): the LPT
assignment, the per-rank shares and the host gather, on the CPU. Two gloo
ranks each take their share of a mixed batch of lists and graphs; the oracle
stands in for the batched GPU calls; rank 0 gathers and the result must equal
the oracle on the whole batch, instance by instance."""
from __future__ import annotations

import os
import socket

import numpy as np
import torch.multiprocessing as mp

import gen
import oracle
from gen import workloads
from paper_1002_4482_gb300 import ranks, shard


def test_lpt_is_greedy_by_decreasing_cost():
    costs = np.array([5, 9, 2, 7, 7, 1, 3])
    parts = shard.lpt_assign(costs, 3)
    load = [int(costs[p].sum()) for p in parts]
    assert sorted(np.concatenate(parts).tolist()) == list(range(len(costs)))
    assert max(load) - min(load) <= costs.max()
    # the classical LPT bound: makespan at most 4/3 of the optimum (lower bound: mean and largest job)
    assert max(load) <= 4 / 3 * max(costs.sum() / 3, costs.max()) + 1e-9
    assert [p.tolist() for p in shard.lpt_assign(costs, 1)] == [list(range(7))]


def test_lpt_is_deterministic_and_balanced_on_the_batch():
    sizes = workloads.batch_sizes(4096)
    for world in (2, 4, 8):
        a = shard.lpt_assign(sizes, world)
        b = shard.lpt_assign(sizes, world)
        assert all(np.array_equal(x, y) for x, y in zip(a, b))
        load = np.array([sizes[p].sum() for p in a])
        assert load.max() / load.mean() < 1.01


def test_shares_and_scatter_back_rebuild_the_batch():
    sizes = gen.loguniform_sizes(31, 0, 9, 5)
    succ, off, heads = gen.list_batch(sizes, 6)
    src, dst, eoff, voff = gen.er_batch(sizes, 2, 1, 7)
    parts = shard.lpt_assign(shard.list_costs(off), 3)
    out = np.full(len(succ), -7, np.int32)
    for idx in parts:
        s, o, h = shard.list_share(succ, off, heads, idx)
        for i, k in enumerate(idx):     # each share is the original lists, in the batched layout
            assert np.array_equal(s[o[i]:o[i + 1]], succ[off[k]:off[k + 1]]) and h[i] == heads[k]
        shard.scatter_back(out, off, idx, oracle.lr_rank_batched(s, o, h))
    assert np.array_equal(out, oracle.lr_rank_batched(succ, off, heads))
    gparts = shard.lpt_assign(shard.graph_costs(eoff, voff), 3)
    lab = np.full(int(voff[-1]), -7, np.int32)
    for idx in gparts:
        a, b, eo, vo = shard.graph_share(src, dst, eoff, voff, idx)
        shard.scatter_back(lab, voff, idx, oracle.cc_batched(a, b, eo, vo))
    assert np.array_equal(lab, oracle.cc_batched(src, dst, eoff, voff))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out: str) -> None:
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    ranks.init("gloo")
    (succ, off, heads), (src, dst, eoff, voff) = workloads.batch(96, 4.0, 12.0, seed=9)
    lparts = shard.lpt_assign(shard.list_costs(off), world)
    gparts = shard.lpt_assign(shard.graph_costs(eoff, voff), world)
    li, gi = lparts[rank], gparts[rank]
    s, o, h = shard.list_share(succ, off, heads, li)
    a, b, eo, vo = shard.graph_share(src, dst, eoff, voff, gi)
    # the oracle stands in for lr_rank_batched / cc_label_batched on this rank's share
    r_part = oracle.lr_rank_batched(s, o, h)
    l_part = oracle.cc_batched(a, b, eo, vo)
    rank_all = shard.gather(r_part, li, off, len(succ))
    lab_all = shard.gather(l_part, gi, voff, int(voff[-1]))
    if rank == 0:
        np.save(out + ".rank.npy", rank_all)
        np.save(out + ".lab.npy", lab_all)
        np.save(out + ".shares.npy", np.array([len(p) for p in lparts] + [len(p) for p in gparts]))
    else:
        assert rank_all is None and lab_all is None
    ranks.shutdown()


def test_two_ranks_gather_equals_the_whole_batch(tmp_path):
    world = 2
    out = str(tmp_path / "res")
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    (succ, off, heads), (src, dst, eoff, voff) = workloads.batch(96, 4.0, 12.0, seed=9)
    rank_all = np.load(out + ".rank.npy")
    lab_all = np.load(out + ".lab.npy")
    shares = np.load(out + ".shares.npy")
    assert shares.min() > 0                       # both ranks had instances of both kinds
    want_r = oracle.lr_rank_batched(succ, off, heads)
    want_l = oracle.cc_batched(src, dst, eoff, voff)
    for k in range(len(off) - 1):                 # instance by instance
        assert np.array_equal(rank_all[off[k]:off[k + 1]], want_r[off[k]:off[k + 1]])
    for k in range(len(voff) - 1):
        assert np.array_equal(lab_all[voff[k]:voff[k + 1]], want_l[voff[k]:voff[k + 1]])
