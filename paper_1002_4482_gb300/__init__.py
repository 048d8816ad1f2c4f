"""GB300-native list ranking and connected components.

Thin Python binding over the C ABI of ``liblrcc.so`` (declared in
``include/lrcc.h``). Every function here only marshals arguments: tensors are
checked for dtype, device and layout, their device pointers and the current
CUDA stream are passed to the C entry point of the same name, and a non-OK
status raises :class:`LrccError`. All computation happens in the CUDA kernels
of ``csrc/``; there is no CPU fallback, and importing the binding on a
machine without the built library raises at first use.

Calls are asynchronous on the current stream. Errors that only the device can
detect (an input that is not a single list, an out-of-range id, a loop that
hit its round cap) are reported by :func:`check` / :func:`last_status`, which
wait for the stream.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "liblrcc.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_NOMEM, ERR_CUDA, ERR_INVALID_INPUT, ERR_NOT_CONVERGED, ERR_TIMEOUT = range(7)
KIND_LR, KIND_LR_WYLLIE, KIND_CC, KIND_LR_BATCH, KIND_CC_BATCH = 1, 2, 3, 4, 5
KIND_CC_SPARSE = 8   # plan class of graphs with fewer than 4 edges per vertex

SYMBOLS = ("lrcc_status_str", "lrcc_version", "lr_rank", "lr_rank_wyllie", "lr_rank_noalloc", "cc_label",
           "lr_rank_host", "cc_label_host", "lr_scan", "lr_scan_forest",
           "lr_rank_batched", "lr_rank_batched_sized", "cc_label_batched", "cc_label_batched_sized", "lrcc_last_status", "lrcc_last_stats",
           "lrcc_wait_check", "lrcc_set_plan", "lrcc_get_plan", "lrcc_reset_plans", "lrcc_release", "lrcc_workspace_bytes",
           "lrcc_workspace_query", "lrcc_set_timing", "lrcc_phase_count", "lrcc_phase_name",
           "lrcc_phase_times", "lrcc_set_l2_fetch_granularity", "lrcc_get_l2_fetch_granularity",
           "lrcc_ctx_create", "lrcc_ctx_reserve", "lrcc_ctx_bytes", "lrcc_ctx_last_status", "lrcc_ctx_destroy",
           "lrcc_gather_probe", "lrcc_chase_probe", "lr_rank_splitters", "lrcc_debug_fail_allocs")


class LrccError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_str(status)} (status {status})")


class Stats(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("levels", ctypes.c_int32),
                ("splitters", ctypes.c_int64 * 8), ("rounds", ctypes.c_int32),
                ("jump_rounds", ctypes.c_int32), ("overflow_chunks", ctypes.c_int64),
                ("edges_read", ctypes.c_int64)]


class Plan(ctypes.Structure):
    _fields_ = [("rs_spacing0", ctypes.c_int32), ("rs_spacing", ctypes.c_int32),
                ("rs_small", ctypes.c_int32), ("rs_chains", ctypes.c_int32),
                ("cc_hook", ctypes.c_int32), ("cc_max_rounds", ctypes.c_int32),
                ("use_graphs", ctypes.c_int32), ("rs_level0", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("cc_sample", ctypes.c_int32)]


def library_path() -> str:
    return _LIB_PATH


def load() -> ctypes.CDLL:
    """Load liblrcc.so (built in-tree by ``__graft_entry__.build()``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"{_LIB_PATH} is missing: build it with __graft_entry__.build()")
        lib = ctypes.CDLL(_LIB_PATH)
        p, i64, i32, i = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
        lib.lrcc_status_str.argtypes = [i]
        lib.lrcc_status_str.restype = ctypes.c_char_p
        lib.lrcc_version.restype = i
        lib.lr_rank.argtypes = [p, i64, i32, p, p]
        lib.lr_rank_wyllie.argtypes = [p, i64, i32, p, p]
        lib.lr_rank_noalloc.argtypes = [p, i64, i32, p, p]
        lib.cc_label.argtypes = [p, p, i64, i64, p, p]
        lib.lr_rank_host.argtypes = [p, i64, i32, p, p]
        lib.lr_scan.argtypes = [p, p, i64, i32, p, p]
        lib.lr_scan_forest.argtypes = [p, p, i64, p, p]
        lib.cc_label_host.argtypes = [p, p, i64, i64, p, p]
        lib.lr_rank_batched.argtypes = [p, p, p, i64, p, p]
        lib.lr_rank_batched_sized.argtypes = [p, p, p, i64, i64, p, p]
        lib.cc_label_batched.argtypes = [p, p, p, p, i64, p, p]
        lib.cc_label_batched_sized.argtypes = [p, p, p, p, i64, i64, p, p]
        lib.lrcc_last_status.argtypes = [p]
        lib.lrcc_wait_check.argtypes = [i, p]
        lib.lrcc_last_stats.argtypes = [p, ctypes.POINTER(Stats)]
        lib.lrcc_set_plan.argtypes = [i, i, i, ctypes.POINTER(Plan)]
        lib.lrcc_get_plan.argtypes = [i, i64, ctypes.POINTER(Plan)]
        lib.lrcc_release.argtypes = [p]
        lib.lrcc_workspace_bytes.restype = i64
        lib.lrcc_workspace_query.argtypes = [i, i64, i64]
        lib.lrcc_workspace_query.restype = i64
        lib.lrcc_set_timing.argtypes = [i]
        lib.lrcc_phase_count.restype = i
        lib.lrcc_phase_name.argtypes = [i]
        lib.lrcc_phase_name.restype = ctypes.c_char_p
        lib.lrcc_phase_times.argtypes = [p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)]
        lib.lrcc_set_l2_fetch_granularity.argtypes = [i]
        lib.lrcc_get_l2_fetch_granularity.restype = i
        lib.lrcc_ctx_create.argtypes = [ctypes.POINTER(p), i]
        lib.lrcc_ctx_reserve.argtypes = [p, p, i64]
        lib.lrcc_ctx_bytes.argtypes = [p]
        lib.lrcc_ctx_bytes.restype = i64
        lib.lrcc_ctx_last_status.argtypes = [p, p]
        lib.lrcc_ctx_destroy.argtypes = [p]
        lib.lrcc_ctx_destroy.restype = None
        lib.lrcc_gather_probe.argtypes = [p, p, i64, p, i64, p, p]
        lib.lrcc_chase_probe.argtypes = [p, i64, i64, i64, p, p]
        lib.lr_rank_splitters.argtypes = [p, i64, i32, p, i64, p, p]
        lib.lrcc_debug_fail_allocs.argtypes = [i]
        lib.lrcc_debug_fail_allocs.restype = i
        for f in ("lr_rank", "lr_rank_wyllie", "lr_rank_noalloc", "cc_label", "lr_rank_host", "cc_label_host",
                  "lr_scan", "lr_scan_forest",
                  "lr_rank_batched",
                  "lr_rank_batched_sized",
                  "cc_label_batched", "cc_label_batched_sized",
                  "lrcc_last_status", "lrcc_last_stats", "lrcc_wait_check", "lrcc_set_plan", "lrcc_get_plan", "lrcc_reset_plans",
                  "lrcc_release", "lrcc_set_timing", "lrcc_phase_times", "lrcc_set_l2_fetch_granularity",
                  "lrcc_ctx_create", "lrcc_ctx_reserve", "lrcc_ctx_last_status", "lrcc_gather_probe",
                  "lrcc_chase_probe", "lr_rank_splitters"):
            getattr(lib, f).restype = i
        _lib = lib
        return lib


def status_str(status: int) -> str:
    return load().lrcc_status_str(int(status)).decode()


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_i32(t: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or t.dtype != torch.int32 or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA int32 tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _dev_i64(t: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or t.dtype != torch.int64 or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA int64 tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _out(out, n, like, name):
    if out is None:
        return torch.empty(n, dtype=torch.int32, device=like.device)
    _dev_i32(out, name)
    if out.numel() != n:
        raise ValueError(f"{name} must hold {n} elements")
    return out


def _host_i32(t: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or t.dtype != torch.int32 or t.is_cuda:
        raise TypeError(f"{name} must be a host (CPU) int32 tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _host_out(out, n, name):
    if out is None:
        return torch.empty(n, dtype=torch.int32, pin_memory=True)
    _host_i32(out, name)
    if out.numel() != n:
        raise ValueError(f"{name} must hold {n} elements")
    return out


def _call(status: int, what: str):
    if status != OK:
        raise LrccError(status, what)


def lr_rank(succ: torch.Tensor, head: int, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Ranks (distance to the tail) of the list stored in ``succ`` (sparse ruling set)."""
    _dev_i32(succ, "succ")
    rank = _out(out, succ.numel(), succ, "out")
    _call(load().lr_rank(succ.data_ptr(), succ.numel(), int(head), rank.data_ptr(), _stream(stream)), "lr_rank")
    return rank


def lr_rank_wyllie(succ: torch.Tensor, head: int, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Same result as :func:`lr_rank`, by Wyllie pointer jumping."""
    _dev_i32(succ, "succ")
    rank = _out(out, succ.numel(), succ, "out")
    _call(load().lr_rank_wyllie(succ.data_ptr(), succ.numel(), int(head), rank.data_ptr(), _stream(stream)),
          "lr_rank_wyllie")
    return rank


def lr_rank_splitters(succ: torch.Tensor, head: int, spl: torch.Tensor, out: torch.Tensor | None = None,
                      stream=None) -> torch.Tensor:
    """Same result as :func:`lr_rank`, with the first-level splitters given
    (spl[0] = head; the paper's even-splitter comparison, Sec. 3.2)."""
    _dev_i32(succ, "succ")
    _dev_i32(spl, "spl")
    rank = _out(out, succ.numel(), succ, "out")
    _call(load().lr_rank_splitters(succ.data_ptr(), succ.numel(), int(head), spl.data_ptr(), spl.numel(),
                                   rank.data_ptr(), _stream(stream)), "lr_rank_splitters")
    return rank


def lr_scan(succ: torch.Tensor, val: torch.Tensor, head: int, out: torch.Tensor | None = None,
            stream=None) -> torch.Tensor:
    """Weighted ranks: sum of ``val`` from each element to the tail, inclusive, modulo 2^32."""
    _dev_i32(succ, "succ")
    _dev_i32(val, "val")
    if val.numel() != succ.numel():
        raise ValueError("val must have one entry per element")
    res = _out(out, succ.numel(), succ, "out")
    _call(load().lr_scan(succ.data_ptr(), val.data_ptr(), succ.numel(), int(head), res.data_ptr(), _stream(stream)),
          "lr_scan")
    return res


def lr_scan_forest(succ: torch.Tensor, val: torch.Tensor, out: torch.Tensor | None = None,
                   stream=None) -> torch.Tensor:
    """:func:`lr_scan` for every list of a forest of lists (no head given)."""
    _dev_i32(succ, "succ")
    _dev_i32(val, "val")
    if val.numel() != succ.numel():
        raise ValueError("val must have one entry per element")
    res = _out(out, succ.numel(), succ, "out")
    _call(load().lr_scan_forest(succ.data_ptr(), val.data_ptr(), succ.numel(), res.data_ptr(), _stream(stream)),
          "lr_scan_forest")
    return res


def lr_rank_noalloc(succ: torch.Tensor, head: int, out: torch.Tensor, stream=None) -> torch.Tensor:
    """Same ranks as :func:`lr_rank` (n <= 2^20) for callers that must not allocate device memory.

    ``out`` must be given (this call allocates nothing); an invalid list sets out[head] = -1."""
    _dev_i32(succ, "succ")
    rank = _out(out, succ.numel(), succ, "out")
    _call(load().lr_rank_noalloc(succ.data_ptr(), succ.numel(), int(head), rank.data_ptr(), _stream(stream)),
          "lr_rank_noalloc")
    return rank


def cc_label(src: torch.Tensor, dst: torch.Tensor, n: int, out: torch.Tensor | None = None,
             stream=None) -> torch.Tensor:
    """Smallest vertex id of each vertex's connected component."""
    _dev_i32(src, "src")
    _dev_i32(dst, "dst")
    if src.numel() != dst.numel():
        raise ValueError("src and dst must have the same length")
    label = _out(out, n, src, "out")
    _call(load().cc_label(src.data_ptr(), dst.data_ptr(), src.numel(), int(n), label.data_ptr(), _stream(stream)),
          "cc_label")
    return label


def lr_rank_host(succ: torch.Tensor, head: int, out: torch.Tensor | None = None, stream=None,
                 sync: bool = True) -> torch.Tensor:
    """:func:`lr_rank` on host tensors: the library copies ``succ`` to the GPU and the ranks back.

    Pinned (page-locked) tensors make the copies asynchronous. With ``sync=False`` the call
    returns once the work is queued on ``stream``; ``out`` is valid (and ``succ`` may change)
    only after the stream is synchronised."""
    _host_i32(succ, "succ")
    rank = _host_out(out, succ.numel(), "out")
    s = _stream(stream)
    _call(load().lr_rank_host(succ.data_ptr(), succ.numel(), int(head), rank.data_ptr(), s), "lr_rank_host")
    if sync:
        (stream or torch.cuda.current_stream()).synchronize()
    return rank


def cc_label_host(src: torch.Tensor, dst: torch.Tensor, n: int, out: torch.Tensor | None = None,
                  stream=None, sync: bool = True) -> torch.Tensor:
    """:func:`cc_label` on host tensors (copies in, labels back); ``sync`` as in :func:`lr_rank_host`."""
    _host_i32(src, "src")
    _host_i32(dst, "dst")
    if src.numel() != dst.numel():
        raise ValueError("src and dst must have the same length")
    label = _host_out(out, n, "out")
    s = _stream(stream)
    _call(load().cc_label_host(src.data_ptr(), dst.data_ptr(), src.numel(), int(n), label.data_ptr(), s),
          "cc_label_host")
    if sync:
        (stream or torch.cuda.current_stream()).synchronize()
    return label


def lr_rank_batched(succ: torch.Tensor, node_off: torch.Tensor, heads: torch.Tensor,
                    out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Ranks of independent lists concatenated in ``succ`` (local ids, int64 offsets).

    The total element count is taken from ``succ.numel()`` (it must equal
    ``node_off[-1]``), so the call does not wait for the stream."""
    _dev_i32(succ, "succ")
    _dev_i64(node_off, "node_off")
    _dev_i32(heads, "heads")
    if node_off.numel() != heads.numel() + 1:
        raise ValueError("node_off must have len(heads) + 1 entries")
    rank = _out(out, succ.numel(), succ, "out")
    _call(load().lr_rank_batched_sized(succ.data_ptr(), node_off.data_ptr(), heads.data_ptr(), heads.numel(),
                                       succ.numel(), rank.data_ptr(), _stream(stream)), "lr_rank_batched")
    return rank


def cc_label_batched(src: torch.Tensor, dst: torch.Tensor, edge_off: torch.Tensor, vert_off: torch.Tensor,
                     n_total: int | None = None, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Min-id component labels of independent graphs (local ids, int64 offsets)."""
    _dev_i32(src, "src")
    _dev_i32(dst, "dst")
    _dev_i64(edge_off, "edge_off")
    _dev_i64(vert_off, "vert_off")
    if edge_off.numel() != vert_off.numel():
        raise ValueError("edge_off and vert_off must have the same length")
    if n_total is None:
        n_total = int(vert_off[-1].item())
    label = _out(out, n_total, src, "out")
    _call(load().cc_label_batched_sized(src.data_ptr(), dst.data_ptr(), edge_off.data_ptr(), vert_off.data_ptr(),
                                        vert_off.numel() - 1, src.numel(), label.data_ptr(), _stream(stream)),
          "cc_label_batched")
    return label


def last_status(stream=None) -> int:
    """Waits for the stream; returns and clears its device status word."""
    return int(load().lrcc_last_status(_stream(stream)))


def wait_check(polls: int, stream=None) -> None:
    """Enqueues the check of the device timeout path (lrcc_wait_check): a bounded
    wait that gives up after `polls` polls and records ERR_TIMEOUT on the stream."""
    _call(load().lrcc_wait_check(int(polls), _stream(stream)), "lrcc_wait_check")


def check(stream=None) -> None:
    """Raises LrccError if the device recorded an error on this stream."""
    st = last_status(stream)
    if st != OK:
        raise LrccError(st, "device")


def last_stats(stream=None) -> dict:
    s = Stats()
    _call(load().lrcc_last_stats(_stream(stream), ctypes.byref(s)), "lrcc_last_stats")
    return {"kind": s.kind, "levels": s.levels, "splitters": list(s.splitters)[: s.levels],
            "rounds": s.rounds, "jump_rounds": s.jump_rounds, "overflow_chunks": s.overflow_chunks,
            "edges_read": s.edges_read}


def set_plan(kind: int, log2_lo: int = 0, log2_hi: int = 32, **fields) -> None:
    p = Plan(**fields)
    _call(load().lrcc_set_plan(kind, log2_lo, log2_hi, ctypes.byref(p)), "lrcc_set_plan")


def set_cc_plan(log2_lo: int = 0, log2_hi: int = 32, **fields) -> None:
    """Plan fields for every components call: graphs with at least 4 edges per
    vertex (KIND_CC) and with fewer (KIND_CC_SPARSE) alike."""
    set_plan(KIND_CC, log2_lo, log2_hi, **fields)
    set_plan(KIND_CC_SPARSE, log2_lo, log2_hi, **fields)


def reset_plans() -> None:
    """Restore the built-in plan table."""
    _call(load().lrcc_reset_plans(), "lrcc_reset_plans")


def get_plan(kind: int, n: int) -> dict:
    p = Plan()
    _call(load().lrcc_get_plan(kind, n, ctypes.byref(p)), "lrcc_get_plan")
    return {f: getattr(p, f) for f, _ in Plan._fields_}


def release(stream=None) -> None:
    _call(load().lrcc_release(_stream(stream)), "lrcc_release")


def workspace_bytes() -> int:
    return int(load().lrcc_workspace_bytes())


def workspace_query(kind: int, n: int, m: int = 0) -> int:
    return int(load().lrcc_workspace_query(kind, n, m))


def gather_probe(src: torch.Tensor, dst: torch.Tensor, table: torch.Tensor, stream=None) -> torch.Tensor:
    """The hook pass's edge stream and two gathers per edge from `table`, without
    the hooking (lrcc_gather_probe): a ceiling for the pass. Returns the device
    int64 sum of the gathered values."""
    src = _dev_i32(src, "src")
    dst = _dev_i32(dst, "dst")
    table = _dev_i32(table, "table")
    out = torch.zeros(1, dtype=torch.int64, device=table.device)
    _call(load().lrcc_gather_probe(src.data_ptr(), dst.data_ptr(), src.numel(), table.data_ptr(), table.numel(),
                                   out.data_ptr(), _stream(stream)), "lrcc_gather_probe")
    return out


def chase_probe(succ: torch.Tensor, chains: int, steps: int, stream=None) -> torch.Tensor:
    """`chains` chains of `steps` dependent reads of succ each, with the first-level
    walk's load form and none of its work (lrcc_chase_probe): a ceiling for the
    walk. Returns the device int64 sum of the elements reached."""
    succ = _dev_i32(succ, "succ")
    out = torch.zeros(1, dtype=torch.int64, device=succ.device)
    _call(load().lrcc_chase_probe(succ.data_ptr(), succ.numel(), int(chains), int(steps), out.data_ptr(),
                                  _stream(stream)), "lrcc_chase_probe")
    return out


def debug_fail_allocs(count: int) -> int:
    """Make the library's next `count` device allocations fail (ERR_NOMEM), for
    testing out-of-memory handling; returns the count that was pending."""
    return int(load().lrcc_debug_fail_allocs(int(count)))


def set_timing(enable: bool) -> None:
    """Phase timing: CUDA events around every kernel (list ranking) or loop (components)."""
    _call(load().lrcc_set_timing(1 if enable else 0), "lrcc_set_timing")


def phase_times(stream=None) -> dict:
    """Waits for the stream; {phase: (total_ms, launches)} recorded since the last query."""
    lib = load()
    k = lib.lrcc_phase_count()
    ms = (ctypes.c_double * k)()
    cnt = (ctypes.c_int64 * k)()
    _call(lib.lrcc_phase_times(_stream(stream), ms, cnt), "lrcc_phase_times")
    return {lib.lrcc_phase_name(i).decode(): (ms[i], cnt[i]) for i in range(k) if cnt[i]}


def set_l2_fetch_granularity(nbytes: int) -> None:
    """L2 fetch unit (32/64/128 B) of the current device's context; affects every kernel."""
    _call(load().lrcc_set_l2_fetch_granularity(int(nbytes)), "lrcc_set_l2_fetch_granularity")


def get_l2_fetch_granularity() -> int:
    return int(load().lrcc_get_l2_fetch_granularity())


class Context:
    """Handle on the library's workspaces of one device (lrcc_ctx_*): reserve a
    stream's workspace ahead of the calls, count the bytes held, free them
    together. The compute calls keep taking a stream."""

    def __init__(self, device: int = 0):
        h = ctypes.c_void_p()
        _call(load().lrcc_ctx_create(ctypes.byref(h), int(device)), "lrcc_ctx_create")
        self._h = h
        self.device = int(device)

    def reserve(self, stream, nbytes: int) -> None:
        _call(load().lrcc_ctx_reserve(self._h, _stream(stream), int(nbytes)), "lrcc_ctx_reserve")

    def bytes(self) -> int:
        return int(load().lrcc_ctx_bytes(self._h))

    def last_status(self, stream=None) -> int:
        return int(load().lrcc_ctx_last_status(self._h, _stream(stream)))

    def close(self) -> None:
        if self._h is not None and self._h.value:
            load().lrcc_ctx_destroy(self._h)
        self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
