"""Host model of the shortcut pass's chases (chase_step in cc_device.cuh): every
vertex chases its parents to the root; a chase longer than QUIET steps stores
the ancestor it has reached in its own vertex's entry at every further step,
so chases passing through that vertex jump ahead. Modelled on a chain of n
links (what the first hook pass leaves on a path of consecutive ids), with
every chase advancing one read per turn: all must end at the root, and with
the progress stores the longest chase takes O(QUIET + log n) reads; without
them about sqrt(2n), because only the final stores of finished chases shorten
the chain, from its root up (n chases of that length are n^1.5 reads in all).
Random forests, chased one read at a time in random orders, must end with
every vertex at its own root."""
from __future__ import annotations

import random

import numpy as np
import pytest

QUIET = 16


def _sync_turns(parent, writes):
    """All chases advance together: in each turn every live chase reads from the
    state the previous turn left, then the turn's stores land (lockstep, as the
    chases of one wave of threads run). Returns the reads each chase took."""
    n = len(parent)
    pos = {v: parent[v] for v in range(n) if parent[v] != v}
    reads = {}
    step = 0
    while pos:
        step += 1
        snap = list(parent)
        stores = {}
        for v, x in list(pos.items()):
            nx = snap[x]
            if nx == x:
                stores[v] = x
                reads[v] = step
                del pos[v]
                continue
            pos[v] = nx
            if writes and step > QUIET:
                stores[v] = nx
        for v, x in stores.items():
            parent[v] = x
    return reads


def _async_random(parent, seed):
    """The same chases with progress stores, one read at a time in a random
    order (stores land at once)."""
    rng = random.Random(seed)
    n = len(parent)
    pos = {v: [parent[v], 0] for v in range(n) if parent[v] != v}
    while pos:
        v = rng.choice(list(pos))
        x, step = pos[v]
        nx = parent[x]
        step += 1
        if nx == x:
            parent[v] = x
            del pos[v]
            continue
        pos[v] = [nx, step]
        if step > QUIET:
            parent[v] = nx


@pytest.mark.parametrize("n", [64, 1024, 4096])
def test_chain_flattens_in_logarithmic_reads(n):
    parent = [max(v - 1, 0) for v in range(n)]
    reads = _sync_turns(parent, writes=True)
    assert parent == [0] * n
    assert max(reads.values()) <= QUIET + 2 * int(np.log2(n)) + 4


def test_chases_without_progress_stores_take_square_root_reads():
    n = 4096
    plain = [max(v - 1, 0) for v in range(n)]
    slow = max(_sync_turns(plain, writes=False).values())
    stored = [max(v - 1, 0) for v in range(n)]
    fast = max(_sync_turns(stored, writes=True).values())
    assert plain == stored == [0] * n
    assert slow >= int(np.sqrt(n)) and slow >= 4 * fast


@pytest.mark.parametrize("seed", range(4))
def test_random_forests_end_at_their_roots_in_any_order(seed):
    # random trees with every link to a smaller id (the only states the hook
    # passes leave), chases advanced in a random order each turn
    rng = np.random.default_rng(seed)
    n = 2000
    parent = [0] * n
    for v in range(n):
        parent[v] = v if rng.random() < 0.05 else int(rng.integers(0, v)) if v else 0
    want = []
    for v in range(n):
        x = v
        while parent[x] != x:
            x = parent[x]
        want.append(x)
    _async_random(parent, seed)
    assert parent == want
