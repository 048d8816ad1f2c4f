"""Checks of the synthetic input generators (no GPU needed)."""
from __future__ import annotations

import numpy as np
import pytest

import gen
import oracle
from gen import workloads


def test_splitmix64_published_values():
    # first outputs of SplitMix64 seeded with 0 (Steele, Lea & Flood 2014; Vigna's C reference)
    assert [gen.splitmix64_at(0, k) for k in (1, 2, 3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_permutation_is_uniform_and_deterministic():
    p = gen.permutation(1000, 7)
    assert np.array_equal(np.sort(p), np.arange(1000))
    assert np.array_equal(p, gen.permutation(1000, 7))
    assert not np.array_equal(p, gen.permutation(1000, 8))
    # position of element 0 over many seeds is roughly uniform over 4 buckets
    pos = np.array([np.flatnonzero(gen.permutation(8, s) == 0)[0] for s in range(4000)])
    counts = np.bincount(pos // 2, minlength=4)
    assert (abs(counts - 1000) < 150).all()


def test_list_random_structure():
    succ, head, perm = gen.list_random(5000, 3, with_perm=True)
    assert head == perm[0]
    assert (succ == -1).sum() == 1
    assert np.array_equal(succ[perm[:-1]], perm[1:])


def test_er_range_and_determinism():
    s, d = gen.er(1000, 100000, 1)
    assert s.min() >= 0 and s.max() < 1000 and d.min() >= 0 and d.max() < 1000
    s2, d2 = gen.er(1000, 100000, 1)
    assert np.array_equal(s, s2) and np.array_equal(d, d2)
    # endpoint counts are close to uniform
    c = np.bincount(s, minlength=1000)
    assert abs(c.mean() - 100) < 1e-9 and c.std() < 15


def test_rmat_quadrant_probabilities():
    scale, m = 10, 200000
    src, dst = gen.rmat(scale, m, 0.57, 0.19, 0.19, 4)
    assert src.min() >= 0 and src.max() < (1 << scale)
    # degree skew: the heaviest vertex is far above the mean degree
    deg = np.bincount(src, minlength=1 << scale) + np.bincount(dst, minlength=1 << scale)
    assert deg.max() > 20 * deg.mean()


def test_batch_generators():
    sizes = workloads.batch_sizes(4096)
    assert sizes.min() >= 256 and sizes.max() < (1 << 20)
    succ, off, heads = gen.list_batch(np.array([3, 1, 5]), 1)
    assert off.tolist() == [0, 3, 4, 9]
    # the permutations returned beside the lists are the order each list is visited in
    s2, o2, h2, perm = gen.list_batch(np.array([3, 1, 5]), 1, with_perm=True)
    assert np.array_equal(s2, succ) and np.array_equal(h2, heads)
    for k in range(3):
        p = perm[off[k]:off[k + 1]]
        assert sorted(p.tolist()) == list(range(off[k + 1] - off[k])) and p[0] == heads[k]
        walk, cur = [], heads[k]
        while cur != -1:
            walk.append(cur)
            cur = succ[off[k] + cur]
        assert walk == p.tolist()
    src, dst, eoff, voff = gen.er_batch(np.array([10, 4]), 2, 1, 1)
    assert eoff.tolist() == [0, 20, 28] and voff.tolist() == [0, 10, 14]
    assert src[:20].max() < 10 and src[20:].max() < 4


def test_jobs_stream():
    arr, kind, size = workloads.serve_jobs(20000, 0.001)
    assert (np.diff(arr) > 0).all()
    assert abs(np.diff(arr).mean() - 0.001) < 0.0001
    assert abs((kind == 0).mean() - 0.7) < 0.02
    assert size.min() >= 1024 and size.max() < (1 << 24)


def test_list_graph_family():
    count, size = 7, 300
    src, dst, n = gen.list_graph(count, size, 3)
    assert n == count * size and len(src) == count * (size - 1)
    ids = np.concatenate([src, dst])
    assert ids.min() >= 0 and ids.max() < n
    # every vertex has degree <= 2, and exactly 2 * count path ends have degree 1
    deg = np.bincount(ids, minlength=n)
    assert deg.max() <= 2 and (deg == 1).sum() == 2 * count and (deg == 0).sum() == 0
    lab = oracle.cc_uf(src, dst, n)
    _, comp_sizes = np.unique(lab, return_counts=True)
    assert len(comp_sizes) == count and (comp_sizes == size).all()


@pytest.mark.parametrize("k", [1, 2, 5])
def test_tree_graph_family(k):
    count, size = 5, 400
    src, dst, n = gen.tree_graph(count, size, k, 4)
    assert n == count * size and len(src) == count * (size - 1)
    # a forest of `count` trees of `size` vertices: n - count edges, count components
    lab = oracle.cc_uf(src, dst, n)
    _, comp_sizes = np.unique(lab, return_counts=True)
    assert len(comp_sizes) == count and (comp_sizes == size).all()
    # edges point child -> parent: every vertex is a child at most once, a parent at most k times
    assert np.bincount(src, minlength=n).max() == 1
    assert np.bincount(dst, minlength=n).max() <= k
    if k == 1:
        assert np.bincount(dst, minlength=n).max() == 1   # degree 1: the trees are paths


def test_density_vertices():
    assert gen.density_vertices(8_000_000, 0.001) == 126492
    n = gen.density_vertices(10_000, 0.01)
    assert abs(10_000 / (n * (n - 1) / 2) - 0.01) < 2e-4


def test_batched_closed_form_matches_oracle():
    # the autotuner checks batched ranks by the generator's closed form; pin
    # that form against the oracle's walk of every list
    import oracle
    from paper_1002_4482_gb300.autotune import _batch_expected_ranks
    sizes = gen.loguniform_sizes(40, 0, 9, 11)
    succ, off, heads, perm = gen.list_batch(sizes, 12, with_perm=True)
    assert np.array_equal(_batch_expected_ranks(off, perm), oracle.lr_rank_batched(succ, off, heads))
