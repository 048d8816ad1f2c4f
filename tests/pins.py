"""Properties that hold for every correct answer, at any size.

List ranking (Sec. 3): the ranks of a single list of n elements are a
permutation of 0..n-1, the tail has rank 0 and every other element ranks one
above its successor.

Connected components (Sec. 4) with min-id labels: both endpoints of an edge
share a label, every label is at most its vertex id, labels are fixed points
(label[label[v]] = label[v]), and no two components share a label, which is
checked by counting: the number of distinct labels equals n minus the number
of successful unions of a spanning forest of the edges. The first three
properties say that every component lies inside one label class and that the
label is the class's smallest member; the count then says that no class holds
two components.
"""
from __future__ import annotations

import numpy as np


def lr_invariants(succ: np.ndarray, head: int, rank: np.ndarray) -> None:
    n = len(succ)
    assert rank.shape == (n,)
    if n == 0:
        return
    assert np.array_equal(np.sort(rank), np.arange(n, dtype=rank.dtype)), "ranks are not a permutation"
    idx = np.arange(n)
    tail = (succ == -1) | (succ == idx)
    assert tail.sum() == 1, "not exactly one tail"
    assert rank[tail][0] == 0, "tail rank is not 0"
    nt = ~tail
    assert np.array_equal(rank[nt], rank[succ[nt]] + 1), "rank[i] != rank[succ[i]] + 1"
    assert rank[head] == n - 1, "head rank is not n-1"


def spanning_forest_unions(src: np.ndarray, dst: np.ndarray, n: int) -> int:
    """Number of edges a spanning forest of the graph keeps (n minus the
    number of components).

    Built by rounds over a forest of parent pointers that always point to a
    smaller id: find every vertex's root (pointer jumping), drop the edges
    whose ends share a root, and give every root that is the larger end of a
    remaining edge the smallest root it meets as its parent. Each root that
    receives a parent joins two different trees, so counting them counts the
    successful unions; each round hooks at least one root, so the rounds end."""
    parent = np.arange(n, dtype=np.int64)
    u = np.asarray(src, np.int64)
    w = np.asarray(dst, np.int64)
    keep = u != w
    u, w = u[keep], w[keep]
    unions = 0
    while len(u):
        while True:
            gp = parent[parent]
            if np.array_equal(gp, parent):
                break
            parent = gp
        ru, rw = parent[u], parent[w]
        diff = ru != rw
        u, w, ru, rw = u[diff], w[diff], ru[diff], rw[diff]
        if len(u) == 0:
            break
        hi, lo = np.maximum(ru, rw), np.minimum(ru, rw)
        best = np.full(n, n, dtype=np.int64)
        np.minimum.at(best, hi, lo)
        hooked = np.flatnonzero(best < n)
        parent[hooked] = best[hooked]
        unions += len(hooked)
    return unions


def cc_invariants(src: np.ndarray, dst: np.ndarray, n: int, label: np.ndarray) -> None:
    assert label.shape == (n,)
    if n == 0:
        return
    v = np.arange(n)
    assert (label >= 0).all() and (label <= v).all(), "label outside [0, v]"
    assert np.array_equal(label[label], label), "labels are not fixed points"
    assert np.array_equal(label[src], label[dst]), "an edge joins two labels"
    classes = len(np.unique(label))
    assert classes == n - spanning_forest_unions(src, dst, n), "a label class holds more than one component"


def lr_sample(succ: np.ndarray, head: int, rank: np.ndarray, samples: int, seed: int) -> None:
    """Exact checks that cost O(samples): rank[i] = rank[succ[i]] + 1 on sampled i,
    rank[head] = n - 1, rank[tail] = 0."""
    n = len(succ)
    rng = np.random.default_rng(seed)
    i = rng.integers(0, n, size=min(samples, n))
    s = succ[i]
    tail = (s == -1) | (s == i)
    assert (rank[i[tail]] == 0).all()
    assert np.array_equal(rank[i[~tail]], rank[s[~tail]] + 1)
    assert rank[head] == n - 1
