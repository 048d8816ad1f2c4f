"""Multi-threaded CPU list ranking by random splitters: a timed baseline on the
host cores (the paper's CPU comparison, Sec. 3.2). Shares no code with the
CUDA library or the oracle; only the benchmark and its tests use it."""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rs_cpu.c")
_LIB = os.path.join(_HERE, "librs_cpu.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    subprocess.run(["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp],
                   check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            p, i64 = ctypes.c_void_p, ctypes.c_int64
            lib.cpu_lr_rank.argtypes = [p, i64, ctypes.c_int32, p, ctypes.c_int, i64, ctypes.c_uint64]
            lib.cpu_lr_rank.restype = ctypes.c_int
            _lib = lib
    return _lib


def lr_rank(succ, head: int, threads: int | None = None, spacing: int = 64, seed: int = 1) -> np.ndarray:
    succ = np.ascontiguousarray(succ, np.int32)
    rank = np.empty(len(succ), np.int32)
    t = threads or os.cpu_count() or 1
    rc = _load().cpu_lr_rank(ctypes.c_void_p(succ.ctypes.data), len(succ), int(head),
                             ctypes.c_void_p(rank.ctypes.data), int(t), int(spacing), int(seed))
    if rc == 4:
        raise ValueError("not a single list")
    if rc:
        raise RuntimeError("cpu_lr_rank failed")
    return rank
