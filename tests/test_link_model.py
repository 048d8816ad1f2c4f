"""Host model of hook rule 5's first pass (link_direct in cc_device.cuh): many
threads link the endpoints of their edges with atomicMin on a parent array
where every vertex starts as its own root, each carrying the link an atomic
displaces on to the next pair. Threads are interleaved one atomic step at a
time in a random order; whatever the order, every edge must end inside one
tree (so the pass joins every edge it reads), no link may point to a larger
id, and the roots must be the oracle's min-id labels."""
from __future__ import annotations

import random

import numpy as np
import pytest

import gen
import oracle


def _link_steps(parent, x, y):
    """One thread's join of x and y, as a generator: each next() performs one
    read or one atomicMin on `parent`, as the device loop does."""
    while x != y:
        hi, lo = max(x, y), min(x, y)
        old = parent[hi]                  # read before the atomic
        yield
        if old > lo:
            old = parent[hi]              # atomicMin returns the value it replaced
            parent[hi] = min(old, lo)
            yield
            if old == hi:
                return
        x, y = old, lo


def _run_pass(n, src, dst, threads, seed):
    parent = list(range(n))
    rng = random.Random(seed)
    work = list(zip(src.tolist(), dst.tolist()))
    per = [work[t::threads] for t in range(threads)]
    active = [[t, None] for t in range(threads)]   # thread, its join in progress
    while active:
        i = rng.randrange(len(active))
        t, g = active[i]
        if g is None:
            if not per[t]:
                active.pop(i)
                continue
            u, v = per[t].pop()
            g = _link_steps(parent, u, v)
            active[i][1] = g
        try:
            next(g)
        except StopIteration:
            active[i][1] = None
    return parent


def _roots(parent):
    out = np.empty(len(parent), np.int64)
    for v in range(len(parent)):
        x = v
        while parent[x] != x:
            x = parent[x]
        out[v] = x
    return out


@pytest.mark.parametrize("seed", range(6))
def test_direct_links_join_every_edge(seed):
    n = 300
    src, dst = gen.er(n, 450, 100 + seed)
    parent = _run_pass(n, src, dst, threads=16, seed=seed)
    assert all(parent[v] <= v for v in range(n))
    roots = _roots(parent)
    assert np.array_equal(roots[src], roots[dst])
    assert np.array_equal(roots.astype(np.int32), oracle.cc_uf(src, dst, n))


def test_direct_links_on_a_path_of_consecutive_ids():
    n = 200
    src = np.arange(n - 1, dtype=np.int32)
    dst = src + 1
    parent = _run_pass(n, dst[::-1].copy(), src[::-1].copy(), threads=8, seed=7)
    assert not _roots(parent).any()


def test_model_detects_a_lost_link():
    # the same model without the carried link (stop after one atomicMin) loses
    # connections on some interleaving, which the checks above would catch
    def one_shot(parent, x, y):
        hi, lo = max(x, y), min(x, y)
        yield
        parent[hi] = min(parent[hi], lo)

    n = 60
    src, dst = gen.er(n, 90, 3)
    lost = False
    for seed in range(20):
        parent = list(range(n))
        rng = random.Random(seed)
        gens = [one_shot(parent, int(u), int(v)) for u, v in zip(src, dst)]
        while gens:
            i = rng.randrange(len(gens))
            try:
                next(gens[i])
            except StopIteration:
                gens.pop(i)
        roots = _roots(parent)
        if not np.array_equal(roots[src], roots[dst]):
            lost = True
            break
    assert lost
