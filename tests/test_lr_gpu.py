"""List-ranking parity: the CUDA path (through the C ABI) against the oracle,
element by element, bit-exact (integers; tolerance 0)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1002_4482_gb300 as lrcc
from gen import workloads
from tests import pins

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
FNS = {"rs": lrcc.lr_rank, "wyllie": lrcc.lr_rank_wyllie}


def _run(fn, succ, head):
    t = torch.from_numpy(np.ascontiguousarray(succ)).to(DEV)
    r = FNS[fn](t, head)
    lrcc.check()
    return r.cpu().numpy()


@pytest.mark.parametrize("fn", ["rs", "wyllie"])
@pytest.mark.parametrize("n", [1, 2, 3, 31, 32, 33, 1000, 8191, 8192, 8193, 16385, 65539, 200003])
def test_random_list_matches_oracle(level0, fn, n):
    for seed in (1, 2):
        succ, head = gen.list_random(n, seed)
        assert np.array_equal(_run(fn, succ, head), oracle.lr_rank(succ, head))


@pytest.mark.parametrize("fn", ["rs", "wyllie"])
def test_list_2p20_matches_oracle(level0, fn):
    succ, head = workloads.lr_random(20)
    assert np.array_equal(_run(fn, succ, head), oracle.lr_rank(succ, head))


@pytest.mark.parametrize("fn", ["rs", "wyllie"])
def test_ordered_and_reversed_layouts(level0, fn):
    n = 100_003
    succ, head = gen.list_ordered(n)
    assert np.array_equal(_run(fn, succ, head), np.arange(n - 1, -1, -1))
    rev = np.arange(-1, n - 1, dtype=np.int32)   # succ[i] = i - 1, head n-1
    assert np.array_equal(_run(fn, rev, n - 1), np.arange(n))


@pytest.mark.parametrize("fn", ["rs", "wyllie"])
def test_selfloop_tail_convention(level0, fn):
    succ, head = gen.list_random(50_000, 3)
    tail = int(np.flatnonzero(succ == -1)[0])
    s2 = succ.copy()
    s2[tail] = tail
    assert np.array_equal(_run(fn, s2, head), oracle.lr_rank(succ, head))


@pytest.mark.parametrize("level0", [1, 2, 3], ids=["inplace", "bucketed", "split"])
def test_result_independent_of_splitters(level0):
    succ, head = gen.list_random(300_000, 4)
    expect = oracle.lr_rank(succ, head)
    base = lrcc.get_plan(lrcc.KIND_LR, 300_000)
    try:
        for seed in (1, 2, 3, 99, 12345):
            for spacing0, spacing, chains, small in ((32, 16, 2, 8192), (4, 4, 1, 1024), (256, 64, 4, 16384),
                                                     (2, 2, 2, 1024)):
                lrcc.set_plan(lrcc.KIND_LR, 0, 32, seed=seed, rs_spacing0=spacing0, rs_spacing=spacing,
                              rs_chains=chains, rs_small=small, rs_level0=level0)
                assert np.array_equal(_run("rs", succ, head), expect), (seed, spacing0, spacing, chains)
    finally:
        lrcc.set_plan(lrcc.KIND_LR, 0, 32, seed=base["seed"])
        _restore_level0()


@pytest.fixture(params=[1, 2, 3], ids=["inplace", "bucketed", "split"])
def level0(request):
    lrcc.set_plan(lrcc.KIND_LR, 0, 32, rs_level0=request.param)
    yield request.param
    _restore_level0()


def _restore_level0():
    # the library's built-in table (see csrc/runtime.cu)
    lrcc.reset_plans()


def test_without_graphs_and_repeated():
    succ, head = gen.list_random(500_000, 5)
    expect = oracle.lr_rank(succ, head)
    t = torch.from_numpy(succ).to(DEV)
    for _ in range(10):
        assert np.array_equal(lrcc.lr_rank(t, head).cpu().numpy(), expect)
    lrcc.set_plan(lrcc.KIND_LR, 0, 32, use_graphs=2)
    lrcc.set_plan(lrcc.KIND_LR_WYLLIE, 0, 32, use_graphs=2)
    try:
        assert np.array_equal(lrcc.lr_rank(t, head).cpu().numpy(), expect)
        assert np.array_equal(lrcc.lr_rank_wyllie(t, head).cpu().numpy(), expect)
    finally:
        lrcc.set_plan(lrcc.KIND_LR, 0, 32, use_graphs=1)
        lrcc.set_plan(lrcc.KIND_LR_WYLLIE, 0, 32, use_graphs=1)
    lrcc.check()


@pytest.mark.parametrize("fn", ["rs", "wyllie"])
def test_unaligned_views(level0, fn):
    # views that start one element into an allocation take the scalar paths
    succ, head = gen.list_random(70_001, 6)
    buf = torch.zeros(70_003, dtype=torch.int32, device=DEV)
    buf[1:70_002] = torch.from_numpy(succ).to(DEV)
    out = torch.zeros(70_003, dtype=torch.int32, device=DEV)
    FNS[fn](buf[1:70_002], head, out=out[1:70_002])
    lrcc.check()
    assert np.array_equal(out[1:70_002].cpu().numpy(), oracle.lr_rank(succ, head))


@pytest.mark.parametrize("fn", ["rs", "wyllie"])
@pytest.mark.parametrize("case", ["cycle", "two_lists", "out_of_range", "shared_successor", "big_cycle"])
def test_invalid_inputs_are_reported(level0, fn, case):
    n = 20_000
    succ, head = gen.list_random(n, 7)
    succ = succ.copy()
    tail = int(np.flatnonzero(succ == -1)[0])
    if case == "cycle":
        succ[tail] = head                          # the whole list becomes a cycle
    elif case == "two_lists":
        succ[succ[head]] = -1                      # cut after the second element
    elif case == "out_of_range":
        succ[tail] = n + 5
    elif case == "shared_successor":
        succ[tail] = succ[head]                    # tail points back into the list
    elif case == "big_cycle":
        mid = succ[succ[succ[head]]]
        succ[tail] = mid
    with pytest.raises(oracle.OracleInvalid):
        oracle.lr_rank(succ, head)
    t = torch.from_numpy(succ).to(DEV)
    FNS[fn](t, head)
    assert lrcc.last_status() == lrcc.ERR_INVALID_INPUT
    # the stream and the library stay usable
    good, h = gen.list_random(n, 8)
    assert np.array_equal(_run(fn, good, h), oracle.lr_rank(good, h))


def test_split_arrays_mark_width_boundary():
    # split first level: 16-bit marks up to 65,534 splitters (indices below the
    # all-ones "not visited" mark), 32-bit marks from 65,535 on
    try:
        for n in (4 * 65534, 4 * 65534 + 1, 4 * 65535, 4 * 65535 + 3, 4 * 65536 + 1):
            lrcc.set_plan(lrcc.KIND_LR, 0, 32, rs_level0=3, rs_spacing0=4, rs_small=1024)
            succ, head = gen.list_random(n, 31)
            assert np.array_equal(_run("rs", succ, head), oracle.lr_rank(succ, head)), n
            assert lrcc.last_stats()["splitters"][0] == (n + 3) // 4
    finally:
        _restore_level0()


def test_host_argument_errors():
    t = torch.zeros(10, dtype=torch.int32, device=DEV)
    with pytest.raises(lrcc.LrccError):
        lrcc.lr_rank(t, 10)
    with pytest.raises(lrcc.LrccError):
        lrcc.lr_rank(t, -1)
    assert lrcc.lr_rank(torch.zeros(0, dtype=torch.int32, device=DEV), 0).numel() == 0


def test_stats_report_levels():
    succ, head = gen.list_random(1 << 22, 9)
    _run("rs", succ, head)
    st = lrcc.last_stats()
    assert st["levels"] >= 1 and st["splitters"][0] > 1
    assert st["splitters"] == sorted(st["splitters"], reverse=True)


def test_overflow_pool_carries_long_sublists():
    # read-only first level with few, long sublists: every walk block's own region
    # (sized for an even share of the elements) overflows into the shared pool,
    # whose segments the scatter then handles as work units of their own
    base = lrcc.get_plan(lrcc.KIND_LR, 1 << 18)
    try:
        for n, spacing0 in ((1 << 18, 4096), (300_007, 1024), (1 << 18, 64)):
            lrcc.set_plan(lrcc.KIND_LR, 0, 32, rs_level0=2, rs_spacing0=spacing0, rs_small=1024)
            succ, head = gen.list_random(n, 21)
            assert np.array_equal(_run("rs", succ, head), oracle.lr_rank(succ, head)), (n, spacing0)
            if spacing0 >= 1024:
                assert lrcc.last_stats()["overflow_chunks"] > 0
    finally:
        lrcc.set_plan(lrcc.KIND_LR, 0, 32, rs_spacing0=base["rs_spacing0"], rs_small=base["rs_small"])
        _restore_level0()


@pytest.mark.parametrize("n", [(1 << 16) + 1, (1 << 17) + 5, 3 * (1 << 20) + 7, (1 << 24) - 3])
def test_read_only_level_ragged_sizes(n):
    # the read-only first level (chunks, bucket scatter, placement) on sizes that
    # leave the last id bucket partial; closed form of the random layout, and the
    # ordered layout, whose walks fill few buckets at a time
    base = lrcc.get_plan(lrcc.KIND_LR, n)
    try:
        lrcc.set_plan(lrcc.KIND_LR, 0, 32, rs_level0=2)
        for seed in (3, 4):
            succ, head, perm = gen.list_random(n, seed, with_perm=True)
            r = _run("rs", succ, head)
            assert np.array_equal(r[perm], np.arange(n - 1, -1, -1, dtype=np.int32)), seed
        succ, head = gen.list_ordered(n)
        assert np.array_equal(_run("rs", succ, head), np.arange(n - 1, -1, -1, dtype=np.int32))
    finally:
        lrcc.set_plan(lrcc.KIND_LR, 0, 32, rs_level0=base["rs_level0"])
        _restore_level0()


@pytest.mark.slow
@pytest.mark.parametrize("n", [(1 << 26) + 12345, (1 << 27) + 777])
def test_read_only_level_large_ragged(n):
    # the default plan's read-only first level between the powers of two the
    # bench uses: random and ordered layouts, closed forms
    succ, head, perm = gen.list_random(n, 5, with_perm=True)
    t = torch.from_numpy(succ).to(DEV)
    rank = lrcc.lr_rank(t, head)
    lrcc.check()
    assert np.array_equal(rank.cpu().numpy()[perm], np.arange(n - 1, -1, -1, dtype=np.int32))
    del t, rank
    succ, head = gen.list_ordered(n)
    rank = lrcc.lr_rank(torch.from_numpy(succ).to(DEV), head)
    lrcc.check()
    assert np.array_equal(rank.cpu().numpy(), np.arange(n - 1, -1, -1, dtype=np.int32))


@pytest.mark.slow
def test_full_size_2p28_random_and_ordered():
    # the bench workload: n = 2^28 in random layout; checked exactly against the
    # generator's closed form rank[perm[k]] = n-1-k and the invariants
    n = 1 << 28
    succ, head, perm = workloads.lr_random(28, with_perm=True)
    t = torch.from_numpy(succ).to(DEV)
    expect = np.arange(n - 1, -1, -1, dtype=np.int32)
    rank = lrcc.lr_rank(t, head)
    lrcc.check()
    r = rank.cpu().numpy()
    assert np.array_equal(r[perm], expect)
    pins.lr_sample(succ, head, r, 1 << 22, 0)
    # the other first-level layouts at the same size: in-place words, split arrays
    try:
        for level0 in (1, 3):
            lrcc.set_plan(lrcc.KIND_LR, 28, 28, rs_level0=level0)
            rank = lrcc.lr_rank(t, head, out=rank)
            lrcc.check()
            assert np.array_equal(rank.cpu().numpy()[perm], expect), level0
    finally:
        _restore_level0()
    del t, rank
    succ, head = workloads.lr_ordered(28)
    rank = lrcc.lr_rank(torch.from_numpy(succ).to(DEV), head)
    lrcc.check()
    assert np.array_equal(rank.cpu().numpy(), np.arange(n - 1, -1, -1, dtype=np.int32))


@pytest.mark.gpu
def test_bounded_wait_records_timeout():
    """The bounded bulk-copy wait gives up on a barrier that no copy completes, records
    ERR_TIMEOUT on the stream and leaves the context usable (a rank call after it is exact)."""
    assert lrcc.last_status() == lrcc.OK
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record()
    lrcc.wait_check(1 << 10)
    ev[1].record()
    assert lrcc.last_status() == lrcc.ERR_TIMEOUT
    assert lrcc.last_status() == lrcc.OK          # read and cleared
    ev[2].record()
    lrcc.wait_check(1 << 14)
    ev[3].record()
    assert lrcc.last_status() == lrcc.ERR_TIMEOUT
    torch.cuda.synchronize()
    print(f"bounded wait: 2^10 polls {ev[0].elapsed_time(ev[1]):.3f} ms, 2^14 polls {ev[2].elapsed_time(ev[3]):.3f} ms")
    with pytest.raises(lrcc.LrccError):
        lrcc.wait_check(0)
    succ, head = gen.list_random(100_003, 5)
    assert np.array_equal(_run("rs", succ, head), oracle.lr_rank(succ, head))


@pytest.mark.parametrize("n", [20_001, 1 << 20, 3_000_017])
def test_given_splitters_even_and_random(n):
    # ranks are the same with the paper's perfect even splitters (list positions
    # 0, D, 2D, ...: sublists of exactly D elements) and with random ones
    succ, head, perm = gen.list_random(n, 41, with_perm=True)
    t = torch.from_numpy(succ).to(DEV)
    expect = np.arange(n - 1, -1, -1, dtype=np.int32)
    for D in (8, 32, 1000):
        even = torch.from_numpy(np.ascontiguousarray(perm[::D])).to(DEV)
        r = lrcc.lr_rank_splitters(t, head, even)
        lrcc.check()
        assert np.array_equal(r.cpu().numpy()[perm], expect), D
        rnd = np.random.default_rng(D).choice(np.arange(1, n), size=(n + D - 1) // D - 1, replace=False)
        spl = np.concatenate([[head], perm[np.sort(rnd)]]).astype(np.int32)
        r = lrcc.lr_rank_splitters(t, head, torch.from_numpy(spl).to(DEV))
        lrcc.check()
        assert np.array_equal(r.cpu().numpy()[perm], expect), D


def test_given_splitters_errors():
    succ, head, perm = gen.list_random(50_000, 42, with_perm=True)
    t = torch.from_numpy(succ).to(DEV)
    for bad in (perm[1::16], np.concatenate([perm[::16], perm[16:17]]), np.concatenate([perm[::16], [60_000]])):
        lrcc.lr_rank_splitters(t, head, torch.from_numpy(np.ascontiguousarray(bad, np.int32)).to(DEV))
        assert lrcc.last_status() == lrcc.ERR_INVALID_INPUT
    with pytest.raises(lrcc.LrccError):
        lrcc.lr_rank_splitters(t, head, torch.zeros(0, dtype=torch.int32, device=DEV))


@pytest.mark.parametrize("n,chains,steps", [(1, 1, 5), (100_003, 1000, 37), (70_001, 4099, 0), (1 << 16, 1 << 14, 300)])
def test_chase_probe_follows_successors(n, chains, steps):
    # on the cyclic list i -> i + 1 (mod n) chain c starts at floor(c n / chains) and
    # reaches start + 1, ..., start + steps (mod n); n = 1 is a self-loop, so every
    # step of its chains restarts at element 0
    succ = ((np.arange(n, dtype=np.int64) + 1) % n).astype(np.int32)
    got = lrcc.chase_probe(torch.from_numpy(succ).to(DEV), chains, steps)
    lrcc.check()
    start = np.arange(chains, dtype=np.int64) * n // chains
    k = np.arange(1, steps + 1, dtype=np.int64)
    want = int(((start[:, None] + k[None, :]) % n).sum()) if n > 1 else 0
    assert int(got.item()) == want


def test_chase_probe_on_a_list_with_a_tail_and_bad_arguments():
    succ, head = gen.list_random(50_000, 9)
    s = torch.from_numpy(succ).to(DEV)
    got = lrcc.chase_probe(s, 2048, 100)
    lrcc.check()
    assert 0 < int(got.item()) <= 2048 * 100 * 49_999
    for chains, steps in ((0, 10), (-1, 10), (10, -1), ((1 << 31) + 1, 1)):
        with pytest.raises(lrcc.LrccError):
            lrcc.chase_probe(s, chains, steps)
