"""Properties that hold for every correct answer, at any size.

List ranking (Sec. 3): the ranks of a single list of n elements are a
permutation of 0..n-1, the tail has rank 0 and every other element ranks one
above its successor.

Connected components (Sec. 4) with min-id labels: both endpoints of an edge
share a label, every label is at most its vertex id, labels are fixed points
(label[label[v]] = label[v]), and every component is connected, which is
checked by counting: the number of distinct labels equals n minus the number
of successful unions of a spanning forest.
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


def cc_invariants(src: np.ndarray, dst: np.ndarray, n: int, label: np.ndarray) -> None:
    assert label.shape == (n,)
    if n == 0:
        return
    v = np.arange(n)
    assert (label >= 0).all() and (label <= v).all(), "label outside [0, v]"
    assert np.array_equal(label[label], label), "labels are not fixed points"
    assert np.array_equal(label[src], label[dst]), "an edge joins two labels"


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
