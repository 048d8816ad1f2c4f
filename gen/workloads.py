"""Named synthetic workloads: the shapes, sizes and seeds used by tests and bench.

The paper draws random lists and random graphs from a seeded generator
(Sec. 3.2 and Sec. 4); these recipes keep that structure and fix the sizes:

* ``lr_random(20)``       one list, n = 2^20, uniformly random layout, seed 1
* ``cc_er(20, 22)``       uniform random multigraph, n = 2^20, m = 2^22, seed 2
* ``lr_random(28)``       one list, n = 2^28, random layout, seed 3
* ``lr_ordered(28)``      the ordered control, succ[i] = i + 1
* ``cc_rmat(24, 16)``     R-MAT, 2^24 vertices, 2^28 edges, (0.57, 0.19, 0.19, 0.05), seed 4
* ``batch(4096)``         2048 lists + 2048 random graphs of average degree 4, sizes
                          log-uniform in [2^8, 2^20), seed 5
* ``serve_jobs(k)``       Poisson stream, 70 % lists / 30 % graphs of average degree 8,
                          sizes log-uniform in [2^10, 2^24), seed 6
"""
from __future__ import annotations

import numpy as np

from . import er, er_batch, jobs, list_batch, list_ordered, list_random, loguniform_sizes, rmat

RMAT_ABC = (0.57, 0.19, 0.19)


def lr_random(log2n: int, seed: int | None = None, with_perm: bool = False):
    if seed is None:
        seed = 1 if log2n <= 24 else 3
    return list_random(1 << log2n, seed, with_perm)


def lr_ordered(log2n: int):
    return list_ordered(1 << log2n)


def cc_er(log2n: int, log2m: int, seed: int = 2):
    n = 1 << log2n
    src, dst = er(n, 1 << log2m, seed)
    return src, dst, n


def cc_rmat(scale: int, edge_factor: int, seed: int = 4):
    n = 1 << scale
    src, dst = rmat(scale, n * edge_factor, *RMAT_ABC, seed)
    return src, dst, n


def batch_sizes(count: int, lo: float = 8.0, hi: float = 20.0, seed: int = 5) -> np.ndarray:
    return loguniform_sizes(count, lo, hi, seed)


def batch(count: int = 4096, lo: float = 8.0, hi: float = 20.0, seed: int = 5, with_perm: bool = False):
    """Half lists (even instance index), half graphs with m = 2n (odd index).
    With ``with_perm`` the list part also carries each list's permutation."""
    sizes = batch_sizes(count, lo, hi, seed)
    lists = list_batch(sizes[0::2], seed * 7919 + 1, with_perm)
    graphs = er_batch(sizes[1::2], 2, 1, seed * 7919 + 2)
    return lists, graphs


def serve_jobs(count: int, mean_gap_s: float, seed: int = 6, lo: float = 10.0, hi: float = 24.0,
               p_list: float = 0.7):
    return jobs(count, mean_gap_s, p_list, lo, hi, seed)
