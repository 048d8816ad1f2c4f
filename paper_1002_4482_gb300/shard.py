"""Batched instances spread over several ranks (one process per GPU).

The instances of a batch are independent, so a batch shards without any
exchange on the data path: a host-side assignment gives every instance to one
rank, each rank runs one batched launch per kind on its share, and the results
come back to one rank with a host gather. Single instances are not sharded.

Assignment: greedy longest-processing-time (LPT). Instances are taken in
decreasing cost and each goes to the rank with the least cost so far (the
lowest rank on ties); the cost of a list is its element count, the cost of a
graph its edge count plus its vertex count. Every rank computes the same
assignment from the same offsets, so no message is needed to agree on it.

Shares keep the batch's layout: a rank's lists (graphs) are concatenated in
the order of their instance index with their own int64 offsets and LOCAL ids,
exactly as the batched calls take them, so results need no relabelling.
"""
from __future__ import annotations

import numpy as np


def lpt_assign(costs: np.ndarray, world: int) -> list[np.ndarray]:
    """Instance indices of each rank, ascending. Greedy LPT over `costs`."""
    costs = np.asarray(costs, np.int64)
    if world < 1:
        raise ValueError("world must be at least 1")
    order = np.argsort(-costs, kind="stable")
    load = np.zeros(world, np.int64)
    owner = np.empty(len(costs), np.int64)
    for k in order:
        r = int(np.argmin(load))          # the first rank with the least load
        owner[k] = r
        load[r] += costs[k]
    return [np.flatnonzero(owner == r) for r in range(world)]


def list_costs(node_off: np.ndarray) -> np.ndarray:
    return np.diff(np.asarray(node_off, np.int64))


def graph_costs(edge_off: np.ndarray, vert_off: np.ndarray) -> np.ndarray:
    return np.diff(np.asarray(edge_off, np.int64)) + np.diff(np.asarray(vert_off, np.int64))


def _take(values: np.ndarray, off: np.ndarray, idx: np.ndarray):
    """The segments idx of a concatenated array, concatenated, with new offsets."""
    off = np.asarray(off, np.int64)
    sizes = off[idx + 1] - off[idx]
    new_off = np.zeros(len(idx) + 1, np.int64)
    np.cumsum(sizes, out=new_off[1:])
    if len(idx) == 0 or new_off[-1] == 0:
        return values[:0].copy(), new_off
    # positions of every kept element in the original array
    starts = np.repeat(off[idx] - new_off[:-1], sizes)
    pos = starts + np.arange(new_off[-1], dtype=np.int64)
    return values[pos], new_off


def list_share(succ: np.ndarray, node_off: np.ndarray, heads: np.ndarray, idx: np.ndarray):
    """(succ, node_off, heads) of the lists idx, in the batched calls' layout."""
    s, off = _take(succ, node_off, idx)
    return s, off, np.asarray(heads)[idx].copy()


def graph_share(src: np.ndarray, dst: np.ndarray, edge_off: np.ndarray, vert_off: np.ndarray, idx: np.ndarray):
    """(src, dst, edge_off, vert_off) of the graphs idx, in the batched calls' layout."""
    a, eoff = _take(src, edge_off, idx)
    b, _ = _take(dst, edge_off, idx)
    vsz = np.diff(np.asarray(vert_off, np.int64))[idx]
    voff = np.zeros(len(idx) + 1, np.int64)
    np.cumsum(vsz, out=voff[1:])
    return a, b, eoff, voff


def scatter_back(out: np.ndarray, off: np.ndarray, idx: np.ndarray, part: np.ndarray) -> None:
    """Writes a rank's concatenated results `part` (instances idx) into `out`,
    the whole batch's result array with offsets `off`."""
    off = np.asarray(off, np.int64)
    sizes = off[idx + 1] - off[idx]
    if sizes.sum() != len(part):
        raise ValueError("a share's results do not match its instances")
    local = np.zeros(len(idx) + 1, np.int64)
    np.cumsum(sizes, out=local[1:])
    pos = np.repeat(off[idx] - local[:-1], sizes) + np.arange(len(part), dtype=np.int64)
    out[pos] = part


def gather(part: np.ndarray, idx: np.ndarray, off: np.ndarray, total: int, dst_rank: int = 0):
    """Host gather of every rank's results to `dst_rank` (torch.distributed,
    object collective over the process group). Returns the whole batch's result
    array on dst_rank and None elsewhere; alone, it returns `part` placed by idx."""
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        out = np.empty(total, part.dtype)
        scatter_back(out, off, idx, part)
        return out
    world = dist.get_world_size()
    me = dist.get_rank()
    got = [None] * world if me == dst_rank else None
    dist.gather_object((idx, part), got, dst=dst_rank)
    if me != dst_rank:
        return None
    out = np.empty(total, part.dtype)
    seen = np.zeros(len(off) - 1, bool)
    for r_idx, r_part in got:
        if seen[r_idx].any():
            raise ValueError("an instance came back from two ranks")
        seen[r_idx] = True
        scatter_back(out, off, r_idx, r_part)
    if not seen.all():
        raise ValueError("an instance came back from no rank")
    return out
