"""Pins for the CPU oracle: it is checked against what the definitions fix,
never against itself or the CUDA path (no GPU needed)."""
from __future__ import annotations

import itertools
import os

import numpy as np
import pytest

import gen
import oracle
from gen import workloads
from tests import pins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out[key] = np.array([int(v) for v in vals], np.int64)
    return out


# ----------------------------------------------------------------- lists --

def test_lr_golden():
    g = _read_golden("lr_small.txt")
    head = int(g["head"][0])
    assert np.array_equal(oracle.lr_rank(g["succ"], head), g["rank"])
    assert np.array_equal(oracle.lr_rank(g["succ_selfloop"], head), g["rank"])


@pytest.mark.parametrize("n", [1, 2, 3, 7, 100, 4096, 65537])
@pytest.mark.parametrize("seed", [1, 17])
def test_lr_closed_form(n, seed):
    # the generator stores the k-th list element at perm[k], so rank[perm[k]] = n-1-k
    succ, head, perm = gen.list_random(n, seed, with_perm=True)
    rank = oracle.lr_rank(succ, head)
    expect = np.empty(n, np.int32)
    expect[perm] = np.arange(n - 1, -1, -1, dtype=np.int32)
    assert np.array_equal(rank, expect)
    pins.lr_invariants(succ, head, rank)


def _distance_to_tail(succ, i):
    d = 0
    while succ[i] != -1 and succ[i] != i:
        i = succ[i]
        d += 1
    return d


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7])
def test_lr_brute_force_all_layouts(n):
    # every storage layout of an n-element list; rank counted by following links
    for order in itertools.permutations(range(n)):
        succ = np.full(n, -1, np.int32)
        for a, b in zip(order, order[1:]):
            succ[a] = b
        rank = oracle.lr_rank(succ, order[0])
        expect = [_distance_to_tail(succ, i) for i in range(n)]
        assert rank.tolist() == expect


def test_lr_ordered_control():
    succ, head = workloads.lr_ordered(12)
    rank = oracle.lr_rank(succ, head)
    assert np.array_equal(rank, np.arange((1 << 12) - 1, -1, -1))


def test_lr_empty():
    assert oracle.lr_rank(np.empty(0, np.int32), 0).shape == (0,)


@pytest.mark.parametrize("succ,head", [
    ([1, 0], 0),                 # cycle, no tail
    ([1, -1, -1], 0),            # two lists
    ([1, 2, 0, -1], 0),          # cycle plus a tail nobody reaches
    ([5, -1], 0),                # successor out of range
    ([2, 2, -1], 0),             # two elements share a successor
])
def test_lr_invalid(succ, head):
    with pytest.raises(oracle.OracleInvalid):
        oracle.lr_rank(np.array(succ, np.int32), head)


def test_lr_pins_reject_mutants():
    # each plausible oracle mistake must break one of the pins used above
    succ, head, perm = gen.list_random(1000, 5, with_perm=True)
    good = oracle.lr_rank(succ, head)
    mutants = [good + 1, (len(succ) - 1) - good, np.roll(good, 1), good[::-1].copy()]
    for bad in mutants:
        with pytest.raises(AssertionError):
            pins.lr_invariants(succ, head, bad)


# ---------------------------------------------------- weighted list ranks --

def test_lr_scan_golden():
    g = _read_golden("lr_scan_small.txt")
    assert np.array_equal(oracle.lr_scan(g["succ"], g["val"], int(g["head"][0])), g["out"])
    assert np.array_equal(oracle.lr_scan_forest(g["forest_succ"], g["forest_val"]), g["forest_out"])


def _suffix_sums_by_layout(perm, val):
    # the k-th list element is stored at perm[k]: out[perm[k]] = sum of val[perm[j]] for j >= k,
    # taken modulo 2^32 by numpy's uint32 arithmetic (a reversed cumulative sum, no walk)
    v = val[perm].astype(np.uint32)
    suf = np.cumsum(v[::-1], dtype=np.uint32)[::-1]
    out = np.empty(len(perm), np.int32)
    out[perm] = suf.view(np.int32)
    return out


@pytest.mark.parametrize("n", [1, 2, 3, 100, 65537])
def test_lr_scan_closed_form(n):
    succ, head, perm = gen.list_random(n, 23, with_perm=True)
    rng = np.random.default_rng(n)
    val = rng.integers(-1000, 1000, n).astype(np.int32)
    assert np.array_equal(oracle.lr_scan(succ, val, head), _suffix_sums_by_layout(perm, val))
    # unit values: one more than the rank (distance to the tail)
    ones = np.ones(n, np.int32)
    expect = np.empty(n, np.int32)
    expect[perm] = np.arange(n, 0, -1, dtype=np.int32)
    assert np.array_equal(oracle.lr_scan(succ, ones, head), expect)


def test_lr_scan_wraps_modulo_2_32():
    n = 1000
    succ, head, perm = gen.list_random(n, 24, with_perm=True)
    val = np.full(n, 2**31 - 7, np.int32)          # the true sums overflow int32 at once
    out = oracle.lr_scan(succ, val, head)
    assert np.array_equal(out, _suffix_sums_by_layout(perm, val))
    k = np.arange(1, n + 1, dtype=np.uint64)
    expect = ((k * (2**31 - 7)) % 2**32).astype(np.uint32).view(np.int32)
    assert np.array_equal(out[perm], expect[::-1])


def _sum_along_path(succ, val, i):
    t = int(val[i])
    while succ[i] != -1 and succ[i] != i:
        i = succ[i]
        t += int(val[i])
    return t


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_lr_scan_brute_force_all_layouts(n):
    # every storage layout, sums by following links from each element
    val = np.array([3, -1, 4, 1, -5, 9][:n], np.int32)
    for order in itertools.permutations(range(n)):
        succ = np.full(n, -1, np.int32)
        for a, b in zip(order, order[1:]):
            succ[a] = b
        out = oracle.lr_scan(succ, val, order[0])
        assert out.tolist() == [_sum_along_path(succ, val, i) for i in range(n)]


@pytest.mark.parametrize("sizes", [[1], [5, 1, 1], [1000, 3, 77, 1, 2], [1] * 50])
def test_lr_scan_forest_closed_form(sizes):
    # a forest: one random permutation cut into consecutive pieces, each piece one list
    n = sum(sizes)
    perm = gen.permutation(n, 25)
    succ = np.full(n, -1, np.int32)
    val = np.random.default_rng(n).integers(-50, 50, n).astype(np.int32)
    expect = np.empty(n, np.int32)
    at = 0
    for sz in sizes:
        piece = perm[at:at + sz]
        succ[piece[:-1]] = piece[1:]
        expect[piece] = _suffix_sums_by_layout(np.arange(sz), val[piece])
        at += sz
    assert np.array_equal(oracle.lr_scan_forest(succ, val), expect)
    # with one piece it is the single-list function
    if len(sizes) == 1:
        assert np.array_equal(oracle.lr_scan(succ, val, int(perm[0])), expect)


def test_lr_scan_brute_force_small_forests():
    # every successor array on 5 elements that forms a forest of lists
    n = 5
    val = np.array([2, -3, 5, 7, 11], np.int32)
    forests = 0
    for succ_t in itertools.product(range(-1, n), repeat=n):
        succ = np.array(succ_t, np.int32)
        named = succ[(succ != -1) & (succ != np.arange(n))]
        # a forest of lists: no element named twice, and no cycle
        ok = len(set(named.tolist())) == len(named)
        if ok:
            for i in range(n):
                j, steps = i, 0
                while succ[j] != -1 and succ[j] != j and steps <= n:
                    j, steps = succ[j], steps + 1
                ok &= steps <= n
        if not ok:
            with pytest.raises(oracle.OracleInvalid):
                oracle.lr_scan_forest(succ, val)
            continue
        forests += 1
        out = oracle.lr_scan_forest(succ, val)
        assert out.tolist() == [_sum_along_path(succ, val, i) for i in range(n)]
    # forests of k labelled lists on 5 elements: Lah number L(5, k); each tail written as -1 or
    # as a self-loop: sum_k L(5, k) 2^k = 120*2 + 240*4 + 120*8 + 20*16 + 1*32
    assert forests == 2512


@pytest.mark.parametrize("succ", [
    [1, 0],                      # cycle
    [2, 2, -1],                  # two predecessors
    [1, 2, 0, -1],               # cycle next to a list
    [5, -1],                     # out of range
])
def test_lr_scan_invalid(succ):
    s = np.array(succ, np.int32)
    v = np.ones(len(succ), np.int32)
    with pytest.raises(oracle.OracleInvalid):
        oracle.lr_scan_forest(s, v)
    with pytest.raises(oracle.OracleInvalid):
        oracle.lr_scan(s, v, 0)
    with pytest.raises(oracle.OracleInvalid):
        oracle.lr_scan(np.array([1, -1, -1], np.int32), np.ones(3, np.int32), 0)   # two lists


def test_lr_scan_pins_reject_mutants():
    # plausible mistakes (exclusive sums, prefix instead of suffix, a lost wrap) fail the closed form
    n = 500
    succ, head, perm = gen.list_random(n, 26, with_perm=True)
    val = np.random.default_rng(3).integers(1, 100, n).astype(np.int32)
    expect = _suffix_sums_by_layout(perm, val)
    exclusive = expect - val
    prefix = np.empty(n, np.int32)
    prefix[perm] = np.cumsum(val[perm])
    for bad in (exclusive, prefix, expect + 1):
        assert not np.array_equal(bad, oracle.lr_scan(succ, val, head))


# ------------------------------------------------------------ components --

def test_cc_golden():
    g = _read_golden("cc_small.txt")
    n = int(g["n"][0])
    for f in (oracle.cc_bfs, oracle.cc_uf):
        assert np.array_equal(f(g["src"], g["dst"], n), g["label"])


def test_cc_brute_force_all_graphs_on_5_vertices():
    n = 5
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        edges = [pairs[b] for b in range(len(pairs)) if mask >> b & 1]
        src = np.array([e[0] for e in edges], np.int32)
        dst = np.array([e[1] for e in edges], np.int32)
        # reachability by boolean closure, label = smallest reachable id
        reach = np.eye(n, dtype=bool)
        for a, b in edges:
            reach[a, b] = reach[b, a] = True
        for k in range(n):
            reach |= reach[:, [k]] & reach[[k], :]
        expect = np.array([np.flatnonzero(reach[v])[0] for v in range(n)])
        assert np.array_equal(oracle.cc_bfs(src, dst, n), expect)
        assert np.array_equal(oracle.cc_uf(src, dst, n), expect)


@pytest.mark.parametrize("k,seg,cycle", [(1, 50, True), (7, 13, False), (40, 25, True), (300, 1, False)])
def test_cc_k_disjoint_segments(k, seg, cycle):
    # k disjoint paths (or cycles) over a random relabelling: exactly k labels,
    # each the smallest id of its segment
    n = k * seg
    relabel = gen.permutation(n, 11)
    src, dst = [], []
    for s in range(k):
        ids = relabel[s * seg:(s + 1) * seg]
        for a, b in zip(ids, ids[1:]):
            src.append(a); dst.append(b)
        if cycle and seg > 2:
            src.append(ids[-1]); dst.append(ids[0])
    src, dst = np.array(src, np.int32), np.array(dst, np.int32)
    order = gen.permutation(len(src), 12)
    src, dst = src[order], dst[order]
    for f in (oracle.cc_bfs, oracle.cc_uf):
        label = f(src, dst, n)
        assert len(np.unique(label)) == k
        for s in range(k):
            ids = relabel[s * seg:(s + 1) * seg]
            assert (label[ids] == ids.min()).all()


def test_cc_matches_scipy():
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    for seed, (n, m) in enumerate([(1000, 600), (5000, 5000), (1 << 14, 1 << 15)]):
        src, dst = gen.er(n, m, 100 + seed)
        a = sp.coo_matrix((np.ones(m), (src, dst)), shape=(n, n))
        ncomp, comp = csgraph.connected_components(a, directed=False)
        first = np.full(ncomp, n, np.int64)
        np.minimum.at(first, comp, np.arange(n))
        expect = first[comp]
        assert np.array_equal(oracle.cc_bfs(src, dst, n), expect)
        assert np.array_equal(oracle.cc_uf(src, dst, n), expect)


def test_cc_bfs_equals_uf_er_and_rmat():
    src, dst = gen.er(1 << 16, 1 << 17, 3)
    a = oracle.cc_bfs(src, dst, 1 << 16)
    assert np.array_equal(a, oracle.cc_uf(src, dst, 1 << 16))
    pins.cc_invariants(src, dst, 1 << 16, a)
    src, dst, n = workloads.cc_rmat(12, 16)
    a = oracle.cc_bfs(src, dst, n)
    assert np.array_equal(a, oracle.cc_uf(src, dst, n))
    pins.cc_invariants(src, dst, n, a)


def test_cc_er_isolated_fraction():
    # each vertex misses all 2m endpoints with probability (1-1/n)^(2m) ~ e^(-2m/n)
    n, m = 1 << 16, 1 << 18
    src, dst = gen.er(n, m, 9)
    label = oracle.cc_uf(src, dst, n)
    deg = np.bincount(src, minlength=n) + np.bincount(dst, minlength=n)
    isolated = (deg == 0).sum()
    expect = n * np.exp(-2 * m / n)
    assert abs(isolated - expect) < 6 * np.sqrt(expect) + 3
    singletons = np.bincount(label, minlength=n)[label] == 1
    assert singletons.sum() >= isolated


def test_spanning_forest_count_matches_scipy():
    # the component count behind cc_invariants, against scipy on graphs with
    # many components, long paths, stars and self-loops
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    cases = [gen.er(3000, 1200, 1), gen.er(500, 5000, 2)]
    s, d, n = gen.list_graph(7, 300, 3)
    cases.append((s, d))
    star = np.arange(1, 400, dtype=np.int32)
    cases.append((star, np.zeros_like(star)))
    cases.append((np.zeros(0, np.int32), np.zeros(0, np.int32)))
    for (s, d), nv in zip(cases, (3000, 500, n, 400, 9)):
        g = coo_matrix((np.ones(len(s)), (s, d)), shape=(nv, nv))
        k = connected_components(g, directed=False)[0]
        assert pins.spanning_forest_unions(s, d, nv) == nv - k


def test_cc_edge_cases():
    e = np.empty(0, np.int32)
    assert np.array_equal(oracle.cc_uf(e, e, 5), np.arange(5))
    assert np.array_equal(oracle.cc_bfs(e, e, 5), np.arange(5))
    assert oracle.cc_uf(e, e, 0).shape == (0,)
    s = np.array([3, 3, 1], np.int32)
    d = np.array([3, 1, 3], np.int32)   # self-loop and duplicate edge
    assert np.array_equal(oracle.cc_uf(s, d, 4), [0, 1, 2, 1])
    with pytest.raises(oracle.OracleInvalid):
        oracle.cc_uf(np.array([0], np.int32), np.array([4], np.int32), 4)


def test_cc_pins_reject_mutants():
    src, dst = gen.er(2000, 1500, 4)
    good = oracle.cc_uf(src, dst, 2000)
    v = np.arange(2000)
    big = np.bincount(good).argmax()
    members = np.flatnonzero(good == big)
    split = good.copy()
    split[members[1:][::2]] = members[1]          # a component broken in two
    zeros = np.zeros(2000, good.dtype)            # every vertex in one class
    roots = np.unique(good)
    a, b = roots[0], roots[1]
    merged = good.copy()
    merged[good == b] = a                         # two components under one label
    mutants = [np.maximum(good, v), v.copy(), split, zeros, merged]
    for bad in mutants:
        with pytest.raises(AssertionError):
            pins.cc_invariants(src, dst, 2000, bad)


# ------------------------------------------------------------- batches --

def test_batched_oracles_match_single():
    sizes = gen.loguniform_sizes(20, 2, 10, 3)
    succ, off, heads = gen.list_batch(sizes, 4)
    rank = oracle.lr_rank_batched(succ, off, heads)
    for k in range(len(sizes)):
        b, e = off[k], off[k + 1]
        assert np.array_equal(rank[b:e], oracle.lr_rank(succ[b:e], heads[k]))
    src, dst, eoff, voff = gen.er_batch(sizes, 2, 1, 5)
    lab = oracle.cc_batched(src, dst, eoff, voff)
    assert np.array_equal(lab, oracle.cc_batched(src, dst, eoff, voff, use_uf=False))
    for k in range(len(sizes)):
        vb, ve, eb, ee = voff[k], voff[k + 1], eoff[k], eoff[k + 1]
        assert np.array_equal(lab[vb:ve], oracle.cc_bfs(src[eb:ee], dst[eb:ee], ve - vb))
