"""CPU oracle (test infrastructure only).

Plain sequential C (``oracle.c``, compiled with gcc on first use) that computes
the definitions of list ranking (Sec. 3) and connected components (Sec. 4).
Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg and the
reference arm of ``bench.py`` may use it; the library never does, and it shares no code with
the CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ARG, INVALID = 0, 1, 4


class OracleInvalid(ValueError):
    """The input is not a valid instance (not a single list, edge out of range)."""


def build(force: bool = False) -> str:
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp],
                   check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            i64, p, i32 = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int32
            lib.oracle_lr_rank.argtypes = [p, i64, i32, p]
            lib.oracle_lr_rank_batched.argtypes = [p, p, p, i64, p]
            lib.oracle_lr_scan.argtypes = [p, p, i64, i32, p]
            lib.oracle_lr_scan_forest.argtypes = [p, p, i64, p]
            lib.oracle_cc_bfs.argtypes = [p, p, i64, i64, p]
            lib.oracle_cc_uf.argtypes = [p, p, i64, i64, p]
            lib.oracle_cc_batched.argtypes = [p, p, p, p, i64, p, ctypes.c_int]
            for f in (lib.oracle_lr_rank, lib.oracle_lr_rank_batched, lib.oracle_lr_scan,
                      lib.oracle_lr_scan_forest, lib.oracle_cc_bfs,
                      lib.oracle_cc_uf, lib.oracle_cc_batched):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def _check(rc: int, what: str):
    if rc == INVALID:
        raise OracleInvalid(what)
    if rc:
        raise ValueError(f"{what}: bad argument")


def lr_rank(succ, head: int) -> np.ndarray:
    """Rank = distance to the tail, by one sequential walk from ``head``."""
    succ = _i32(succ)
    rank = np.empty(len(succ), np.int32)
    _check(_load().oracle_lr_rank(_p(succ), len(succ), int(head), _p(rank)), "lr_rank")
    return rank


def lr_scan(succ, val, head: int) -> np.ndarray:
    """Weighted ranks: sum of val from each element to its tail, inclusive, modulo 2^32."""
    succ, val = _i32(succ), _i32(val)
    out = np.empty(len(succ), np.int32)
    _check(_load().oracle_lr_scan(_p(succ), _p(val), len(succ), int(head), _p(out)), "lr_scan")
    return out


def lr_scan_forest(succ, val) -> np.ndarray:
    """lr_scan for every list of a forest of lists (heads found by in-degree)."""
    succ, val = _i32(succ), _i32(val)
    out = np.empty(len(succ), np.int32)
    _check(_load().oracle_lr_scan_forest(_p(succ), _p(val), len(succ), _p(out)), "lr_scan_forest")
    return out


def lr_rank_batched(succ, node_off, heads) -> np.ndarray:
    succ, heads = _i32(succ), _i32(heads)
    off = np.ascontiguousarray(node_off, np.int64)
    rank = np.empty(len(succ), np.int32)
    _check(_load().oracle_lr_rank_batched(_p(succ), _p(off), _p(heads), len(heads), _p(rank)),
           "lr_rank_batched")
    return rank


def cc_bfs(src, dst, n: int) -> np.ndarray:
    """Component label = smallest vertex id, by BFS in increasing start order."""
    src, dst = _i32(src), _i32(dst)
    label = np.empty(n, np.int32)
    _check(_load().oracle_cc_bfs(_p(src), _p(dst), len(src), n, _p(label)), "cc_bfs")
    return label


def cc_uf(src, dst, n: int) -> np.ndarray:
    """Component label = smallest vertex id, by union-find with min-id roots."""
    src, dst = _i32(src), _i32(dst)
    label = np.empty(n, np.int32)
    _check(_load().oracle_cc_uf(_p(src), _p(dst), len(src), n, _p(label)), "cc_uf")
    return label


def cc_label(src, dst, n: int) -> np.ndarray:
    return cc_uf(src, dst, n)


def cc_batched(src, dst, edge_off, vert_off, use_uf: bool = True) -> np.ndarray:
    src, dst = _i32(src), _i32(dst)
    eoff = np.ascontiguousarray(edge_off, np.int64)
    voff = np.ascontiguousarray(vert_off, np.int64)
    label = np.empty(int(voff[-1]), np.int32)
    _check(_load().oracle_cc_batched(_p(src), _p(dst), _p(eoff), _p(voff), len(voff) - 1,
                                     _p(label), int(use_uf)), "cc_batched")
    return label
