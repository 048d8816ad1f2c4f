"""Connected-components parity: the CUDA path (through the C ABI) against the
oracle, element by element, bit-exact (min-id labels are unique)."""
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


def _run(src, dst, n):
    s = torch.from_numpy(np.ascontiguousarray(src, np.int32)).to(DEV)
    d = torch.from_numpy(np.ascontiguousarray(dst, np.int32)).to(DEV)
    lab = lrcc.cc_label(s, d, n)
    lrcc.check()
    return lab.cpu().numpy()


@pytest.fixture(params=[1, 2, 3, 4, 5],
                ids=["hook-once", "hook-relink", "hook-once-then-relink", "shiloach-vishkin", "link-first-pass"])
def hook(request):
    lrcc.set_cc_plan(0, 32, cc_hook=request.param)
    yield request.param
    lrcc.reset_plans()


@pytest.mark.parametrize("n,m", [(1, 0), (1, 1), (5, 0), (10, 3), (33, 40), (1000, 500), (1000, 3000),
                                 (1 << 14, 1 << 15), (100_003, 150_001)])
def test_er_matches_oracle(hook, n, m):
    for seed in (1, 2):
        src, dst = gen.er(n, m, seed)
        assert np.array_equal(_run(src, dst, n), oracle.cc_bfs(src, dst, n))


def test_er_2p20_2p22_matches_oracle(hook):
    src, dst, n = workloads.cc_er(20, 22)
    lab = _run(src, dst, n)
    assert np.array_equal(lab, oracle.cc_uf(src, dst, n))
    st = lrcc.last_stats()
    assert st["rounds"] >= 2


def test_rmat_scale16_matches_oracle(hook):
    src, dst, n = workloads.cc_rmat(16, 16)
    assert np.array_equal(_run(src, dst, n), oracle.cc_uf(src, dst, n))


@pytest.mark.parametrize("k,seg,cycle", [(1, 100_000, False), (1, 99_999, True), (64, 1000, True),
                                         (3000, 7, False)])
def test_paths_and_cycles(hook, k, seg, cycle):
    # long paths are the slow case for hooking (Sec. 4: lists take many rounds)
    n = k * seg
    relabel = gen.permutation(n, 21)
    ids = relabel.reshape(k, seg)
    src = ids[:, :-1].ravel()
    dst = ids[:, 1:].ravel()
    if cycle:
        src = np.concatenate([src, ids[:, -1]])
        dst = np.concatenate([dst, ids[:, 0]])
    order = gen.permutation(len(src), 22)
    lab = _run(src[order], dst[order], n)
    assert np.array_equal(lab, oracle.cc_uf(src, dst, n))
    assert len(np.unique(lab)) == k


@pytest.mark.parametrize("k,seg,reverse", [(1, 1 << 22, False), (1, 1 << 20, True), (256, 4096, False)])
def test_paths_of_consecutive_ids(hook, k, seg, reverse):
    # k paths whose edges join consecutive ids, in id order (a 1-D chain): the first
    # hook pass hangs every vertex below its predecessor, one chain per path as deep
    # as the path is long, which the shortcut then has to flatten; labels are each
    # path's first id (closed form)
    n = k * seg
    ids = np.arange(n, dtype=np.int64).reshape(k, seg)
    src = ids[:, :-1].ravel().astype(np.int32)
    dst = ids[:, 1:].ravel().astype(np.int32)
    if reverse:
        src, dst = dst[::-1].copy(), src[::-1].copy()
    lab = _run(src, dst, n)
    assert np.array_equal(lab, np.repeat(ids[:, 0], seg).astype(np.int32))


def test_self_loops_duplicates_isolated(hook):
    src = np.array([3, 3, 3, 7, 7, 1], np.int32)
    dst = np.array([3, 5, 5, 7, 5, 1], np.int32)
    assert _run(src, dst, 9).tolist() == [0, 1, 2, 3, 4, 3, 6, 3, 8]


def test_graphs_off_and_repeated(hook):
    src, dst = gen.er(200_000, 300_000, 3)
    expect = oracle.cc_uf(src, dst, 200_000)
    for _ in range(5):
        assert np.array_equal(_run(src, dst, 200_000), expect)
    lrcc.set_cc_plan(0, 32, use_graphs=2)
    try:
        assert np.array_equal(_run(src, dst, 200_000), expect)
    finally:
        lrcc.set_cc_plan(0, 32, use_graphs=1)


def test_unaligned_views():
    src, dst = gen.er(10_001, 20_003, 4)
    s = torch.zeros(20_005, dtype=torch.int32, device=DEV)
    d = torch.zeros(20_005, dtype=torch.int32, device=DEV)
    s[1:20_004] = torch.from_numpy(src).to(DEV)
    d[1:20_004] = torch.from_numpy(dst).to(DEV)
    out = torch.zeros(10_003, dtype=torch.int32, device=DEV)
    lrcc.cc_label(s[1:20_004], d[1:20_004], 10_001, out=out[1:10_002])
    lrcc.check()
    assert np.array_equal(out[1:10_002].cpu().numpy(), oracle.cc_uf(src, dst, 10_001))


def test_out_of_range_edge_is_reported():
    src = np.array([0, 1, 2], np.int32)
    dst = np.array([1, 2, 9], np.int32)
    s, d = torch.from_numpy(src).to(DEV), torch.from_numpy(dst).to(DEV)
    lrcc.cc_label(s, d, 5)
    assert lrcc.last_status() == lrcc.ERR_INVALID_INPUT
    assert _run(src[:2], dst[:2], 5).tolist() == [0, 0, 0, 3, 4]


def test_round_cap_is_reported():
    # with a cap of one pass, any graph whose first pass joins two trees must
    # stop with NOT_CONVERGED; the default cap then labels it correctly
    src, dst = gen.er(5000, 4000, 5)
    s, d = torch.from_numpy(src).to(DEV), torch.from_numpy(dst).to(DEV)
    lrcc.set_cc_plan(0, 32, cc_max_rounds=1)
    try:
        lrcc.cc_label(s, d, 5000)
        st = lrcc.last_status()
    finally:
        lrcc.set_cc_plan(0, 32, cc_max_rounds=-1)
    assert st == lrcc.ERR_NOT_CONVERGED
    assert lrcc.get_plan(lrcc.KIND_CC, 5000)["cc_max_rounds"] == 0
    assert lrcc.get_plan(lrcc.KIND_CC_SPARSE, 5000)["cc_max_rounds"] == 0
    assert np.array_equal(_run(src, dst, 5000), oracle.cc_uf(src, dst, 5000))


@pytest.mark.parametrize("sample", [1, 2, 8, 64, -1], ids=["off", "half", "eighth", "1/64", "auto"])
def test_sample_pass_keeps_labels(hook, sample):
    # the sample pass hooks a prefix of the edge list first; labels must not change,
    # whatever the prefix holds: dense random graphs, many small components, a
    # prefix that already holds every edge (the list repeated), and a long path
    # whose prefix is one piece of it
    lrcc.set_cc_plan(0, 32, cc_sample=sample)
    try:
        src, dst = gen.er(1 << 16, 1 << 20, 41)           # 16 edges per vertex
        assert np.array_equal(_run(src, dst, 1 << 16), oracle.cc_uf(src, dst, 1 << 16))
        src, dst = gen.er(1 << 17, 1 << 17, 42)           # one edge per vertex: small components
        assert np.array_equal(_run(src, dst, 1 << 17), oracle.cc_uf(src, dst, 1 << 17))
        s1, d1 = gen.er(50_000, 20_000, 43)
        src, dst = np.tile(s1, 8), np.tile(d1, 8)          # the prefix is the whole edge set
        assert np.array_equal(_run(src, dst, 50_000), oracle.cc_uf(s1, d1, 50_000))
        n = 300_000
        relabel = gen.permutation(n, 44)
        src = relabel[:-1].astype(np.int32)
        dst = relabel[1:].astype(np.int32)                 # one path, edges in path order
        assert np.array_equal(_run(src, dst, n), oracle.cc_uf(src, dst, n))
        src, dst, n = workloads.cc_rmat(16, 16)
        assert np.array_equal(_run(src, dst, n), oracle.cc_uf(src, dst, n))
    finally:
        lrcc.set_cc_plan(0, 32, cc_hook=hook, cc_sample=-1)


def test_stats_count_edges_read():
    # no sample pass: the first pass reads every edge, each later pass at most all of them;
    # with the sample pass of m/16 edges, that prefix is read once more
    src, dst = gen.er(1 << 16, 1 << 20, 45)
    try:
        for sample, extra in ((1, 0), (16, (1 << 20) // 16)):
            lrcc.set_cc_plan(0, 32, cc_sample=sample, cc_hook=1)
            assert np.array_equal(_run(src, dst, 1 << 16), oracle.cc_uf(src, dst, 1 << 16))
            st = lrcc.last_stats()
            assert (1 << 20) + extra <= st["edges_read"] <= st["rounds"] * (1 << 20) + extra, (sample, st)
    finally:
        lrcc.reset_plans()


@pytest.mark.parametrize("family", ["lists", "trees-2", "trees-5", "trees-20", "density-0.001", "density-0.01"])
def test_paper_graph_families(hook, family):
    # the families of the paper's component experiments (Sec. 4): collections of
    # random lists, random trees of degree k, random graphs of edge density d;
    # labels against the oracle, and the Shiloach-Vishkin rounds within their
    # bound floor(log_{3/2} n) + 2
    m = 200_000
    if family == "lists":
        src, dst, n = gen.list_graph(4, m // 4 + 1, 51)
    elif family.startswith("trees"):
        k = int(family.split("-")[1])
        src, dst, n = gen.tree_graph(4, m // 4 + 1, k, 52)
    else:
        d = float(family.split("-")[1])
        n = gen.density_vertices(m, d)
        src, dst = gen.er(n, m, 53)
    assert np.array_equal(_run(src, dst, n), oracle.cc_uf(src, dst, n))
    if hook == 4:
        bound = int(np.floor(np.log(n) / np.log(1.5))) + 2
        assert lrcc.last_stats()["rounds"] <= bound


@pytest.mark.slow
def test_full_size_rmat_scale24(hook):
    # the bench workload: R-MAT 2^24 vertices, 2^28 edges, against the union-find oracle
    src, dst, n = workloads.cc_rmat(24, 16)
    lab = _run(src, dst, n)
    # cheap properties first (the count of components needs every edge, so the
    # exact comparison below stands in for it)
    assert (lab <= np.arange(n)).all() and np.array_equal(lab[lab], lab)
    assert np.array_equal(lab[src[: 1 << 24]], lab[dst[: 1 << 24]])
    assert np.array_equal(lab, oracle.cc_uf(src, dst, n))


def test_gather_probe_reads_every_endpoint():
    # the hook pass's ceiling probe gathers table[src[e]] + table[dst[e]] for every edge
    n, m = 5000, 40_003
    src, dst = gen.er(n, m, 61)
    table = np.random.default_rng(3).integers(0, 1 << 30, n).astype(np.int32)
    got = lrcc.gather_probe(torch.from_numpy(src).to(DEV), torch.from_numpy(dst).to(DEV),
                            torch.from_numpy(table).to(DEV))
    lrcc.check()
    want = int(table[src].astype(np.int64).sum() + table[dst].astype(np.int64).sum())
    assert int(got.item()) == want


@pytest.mark.slow
def test_large_sparse_graph_takes_its_plan_class():
    # 2^24 + 1000 vertices, 2 edges per vertex: the sparse class's built-in plan
    # for 2^25 (re-linking after a sample pass) against union-find
    n = (1 << 24) + 1000
    src, dst = gen.er(n, 2 * n, 71)
    assert lrcc.get_plan(lrcc.KIND_CC_SPARSE, n)["cc_hook"] == 3
    assert np.array_equal(_run(src, dst, n), oracle.cc_uf(src, dst, n))
    src, dst, n2 = gen.list_graph(64, (1 << 24) // 64 + 3, 72)     # long paths: many passes
    assert np.array_equal(_run(src, dst, n2), oracle.cc_uf(src, dst, n2))
