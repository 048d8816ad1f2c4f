"""Seeded synthetic inputs for list ranking and connected components.

The generators live in ``gen.c`` (compiled on first use with gcc) and hold
none of the ranking or labelling arithmetic; the CPU oracle and the CUDA path
are both fed from here. Every array is a numpy array of the dtype the library
takes: int32 node/vertex ids, int64 offsets.

Workload recipes (sizes, seeds, distributions) are in :mod:`gen.workloads`.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into libgen.so (OpenMP when the compiler has it)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:5] + ["-fopenmp"] + base[5:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            i64, u64, p = ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p
            dbl = ctypes.c_double
            lib.gen_permutation.argtypes = [i64, u64, p]
            lib.gen_list_random.argtypes = [i64, u64, p, p, p]
            lib.gen_list_random.restype = ctypes.c_int
            lib.gen_list_ordered.argtypes = [i64, p, p]
            lib.gen_er.argtypes = [i64, i64, u64, p, p]
            lib.gen_rmat.argtypes = [ctypes.c_int, i64, dbl, dbl, dbl, u64, p, p]
            lib.gen_rmat.restype = ctypes.c_int
            lib.gen_loguniform_sizes.argtypes = [i64, dbl, dbl, u64, p]
            lib.gen_list_batch.argtypes = [i64, p, u64, p, p, p, p]
            lib.gen_list_batch.restype = ctypes.c_int
            lib.gen_er_batch.argtypes = [i64, p, i64, i64, u64, p, p, p, p]
            lib.gen_jobs.argtypes = [i64, dbl, dbl, dbl, dbl, u64, p, p, p]
            lib.gen_list_graph.argtypes = [i64, i64, u64, p, p]
            lib.gen_list_graph.restype = ctypes.c_int
            lib.gen_tree_graph.argtypes = [i64, i64, i64, u64, p, p]
            lib.gen_tree_graph.restype = ctypes.c_int
            lib.gen_splitmix64_at.argtypes = [u64, u64]
            lib.gen_splitmix64_at.restype = u64
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def permutation(n: int, seed: int) -> np.ndarray:
    lib = _load()
    p = np.empty(n, np.int32)
    lib.gen_permutation(n, seed, _ptr(p))
    return p


def list_random(n: int, seed: int, with_perm: bool = False):
    """Random-layout list: returns (succ, head) or (succ, head, perm)."""
    lib = _load()
    succ = np.empty(n, np.int32)
    head = ctypes.c_int32(-1)
    perm = np.empty(n, np.int32) if with_perm else None
    rc = lib.gen_list_random(n, seed, _ptr(succ), ctypes.byref(head), _ptr(perm))
    if rc:
        raise MemoryError("gen_list_random failed")
    return (succ, head.value, perm) if with_perm else (succ, head.value)


def list_ordered(n: int):
    lib = _load()
    succ = np.empty(n, np.int32)
    head = ctypes.c_int32(-1)
    lib.gen_list_ordered(n, _ptr(succ), ctypes.byref(head))
    return succ, head.value


def er(n: int, m: int, seed: int):
    lib = _load()
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    lib.gen_er(n, m, seed, _ptr(src), _ptr(dst))
    return src, dst


def rmat(scale: int, m: int, a: float, b: float, c: float, seed: int):
    lib = _load()
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    if lib.gen_rmat(scale, m, a, b, c, seed, _ptr(src), _ptr(dst)):
        raise ValueError("gen_rmat failed")
    return src, dst


def list_graph(count: int, size: int, seed: int):
    """count paths of `size` vertices at random ids: (src, dst, n)."""
    lib = _load()
    m = count * max(size - 1, 0)
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    if lib.gen_list_graph(count, size, seed, _ptr(src), _ptr(dst)):
        raise MemoryError("gen_list_graph failed")
    return src, dst, count * size


def tree_graph(count: int, size: int, k: int, seed: int):
    """count random trees of `size` vertices, at most k children each: (src, dst, n)."""
    lib = _load()
    m = count * max(size - 1, 0)
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    if lib.gen_tree_graph(count, size, k, seed, _ptr(src), _ptr(dst)):
        raise MemoryError("gen_tree_graph failed")
    return src, dst, count * size


def density_vertices(m: int, d: float) -> int:
    """Vertex count n of a graph with m edges and edge density d = m / (n (n - 1) / 2)."""
    return int(round((1.0 + (1.0 + 8.0 * m / d) ** 0.5) / 2.0))


def loguniform_sizes(count: int, lo: float, hi: float, seed: int) -> np.ndarray:
    lib = _load()
    s = np.empty(count, np.int64)
    lib.gen_loguniform_sizes(count, lo, hi, seed, _ptr(s))
    return s


def list_batch(sizes: np.ndarray, seed: int, with_perm: bool = False):
    """Concatenated random lists: returns (succ, node_off, heads), local ids,
    plus, with ``with_perm``, the concatenated per-list permutations (list k
    visits perm[node_off[k]], perm[node_off[k] + 1], ... in local ids)."""
    lib = _load()
    sizes = np.ascontiguousarray(sizes, np.int64)
    count = len(sizes)
    off = np.empty(count + 1, np.int64)
    succ = np.empty(int(sizes.sum()), np.int32)
    heads = np.empty(count, np.int32)
    perm = np.empty(len(succ), np.int32) if with_perm else None
    if lib.gen_list_batch(count, _ptr(sizes), seed, _ptr(off), _ptr(succ), _ptr(heads), _ptr(perm)):
        raise MemoryError("gen_list_batch failed")
    return (succ, off, heads, perm) if with_perm else (succ, off, heads)


def er_batch(vsizes: np.ndarray, deg_num: int, deg_den: int, seed: int):
    """Concatenated random graphs: returns (src, dst, edge_off, vert_off), local ids."""
    lib = _load()
    vsizes = np.ascontiguousarray(vsizes, np.int64)
    count = len(vsizes)
    voff = np.empty(count + 1, np.int64)
    eoff = np.empty(count + 1, np.int64)
    lib.gen_er_batch(count, _ptr(vsizes), deg_num, deg_den, seed, _ptr(voff), _ptr(eoff), None, None)
    m = int(eoff[-1])
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    lib.gen_er_batch(count, _ptr(vsizes), deg_num, deg_den, seed, _ptr(voff), _ptr(eoff), _ptr(src), _ptr(dst))
    return src, dst, eoff, voff


def jobs(count: int, mean_gap: float, p_list: float, lo: float, hi: float, seed: int):
    """Poisson job stream: returns (arrival_s, kind, size); kind 0 = list, 1 = graph."""
    lib = _load()
    arr = np.empty(count, np.float64)
    kind = np.empty(count, np.int32)
    size = np.empty(count, np.int64)
    lib.gen_jobs(count, mean_gap, p_list, lo, hi, seed, _ptr(arr), _ptr(kind), _ptr(size))
    return arr, kind, size


def splitmix64_at(seed: int, k: int) -> int:
    return int(_load().gen_splitmix64_at(seed, k))
