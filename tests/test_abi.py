"""The C-ABI library loads and exports every function include/lrcc.h declares
(no GPU needed; no compute call is made)."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

import paper_1002_4482_gb300 as lrcc
from paper_1002_4482_gb300 import _build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "lrcc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b([a-z_][a-z0-9_]*)\s*\(", text)
    skip = {"if", "for", "while", "return", "sizeof", "defined"}
    return sorted({n for n in names if n not in skip and not n.startswith("__")})


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return ctypes.CDLL(_build.OUT)


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("lr_rank", "lr_rank_wyllie", "cc_label", "lr_rank_batched", "cc_label_batched",
              "lrcc_last_status"):
        assert f in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"liblrcc.so does not export {name}"


def test_binding_names_match_header():
    assert set(lrcc.SYMBOLS) == set(declared_functions())


def declared_arity():
    """Parameter count of every function prototype in the header."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for name, params in re.findall(r"\b([a-z_][a-z0-9_]*)\s*\(([^()]*)\)\s*;", text):
        params = params.strip()
        out[name] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_declares_argument_types_for_every_call():
    # a ctypes call without argtypes passes Python ints as 32-bit C ints, which
    # truncates 64-bit pointers and sizes: every function with parameters needs them
    L = lrcc.load()
    for name, k in declared_arity().items():
        if k == 0:
            continue
        at = getattr(L, name).argtypes
        assert at is not None and len(at) == k, f"{name}: argtypes {at} for {k} parameters"


def test_status_strings(lib):
    lrcc.load()
    assert lrcc.status_str(0) == "ok"
    assert "invalid input" in lrcc.status_str(4)
    assert lrcc.status_str(99) == "unknown status"
    assert lrcc.load().lrcc_version() == 101


def test_host_side_argument_errors_need_no_gpu(lib):
    # rejected before any CUDA call: negative size, head out of range, NULL pointers
    L = lrcc.load()
    assert L.lr_rank(None, -1, 0, None, None) == lrcc.ERR_ARG
    assert L.lr_rank(None, 0, 0, None, None) == lrcc.OK
    assert L.lr_rank(ctypes.c_void_p(16), 10, 10, ctypes.c_void_p(16), None) == lrcc.ERR_ARG
    assert L.lr_rank(None, 10, 0, None, None) == lrcc.ERR_ARG
    assert L.lr_rank_wyllie(None, 5, -1, None, None) == lrcc.ERR_ARG
    assert L.cc_label(None, None, 0, 0, None, None) == lrcc.OK
    assert L.cc_label(None, None, 5, 0, None, None) == lrcc.ERR_ARG
    assert L.cc_label(None, None, 0, 5, None, None) == lrcc.ERR_ARG
    assert L.lr_rank_batched(None, None, None, 0, None, None) == lrcc.OK
    assert L.cc_label_batched(None, None, None, None, -1, None, None) == lrcc.ERR_ARG
    # measurement aids: sizes and pointers checked before the stream's state is touched
    p16 = ctypes.c_void_p(16)
    assert L.lrcc_chase_probe(p16, 0, 1, 1, p16, None) == lrcc.ERR_ARG
    assert L.lrcc_chase_probe(p16, 1 << 31, 1, 1, p16, None) == lrcc.ERR_ARG
    assert L.lrcc_chase_probe(p16, 10, 0, 1, p16, None) == lrcc.ERR_ARG
    assert L.lrcc_chase_probe(p16, 10, (1 << 31) + 1, 1, p16, None) == lrcc.ERR_ARG
    assert L.lrcc_chase_probe(p16, 10, 4, -1, p16, None) == lrcc.ERR_ARG
    assert L.lrcc_chase_probe(None, 10, 4, 1, p16, None) == lrcc.ERR_ARG
    assert L.lrcc_chase_probe(p16, 10, 4, 1, None, None) == lrcc.ERR_ARG
    assert L.lrcc_gather_probe(p16, p16, -1, p16, 10, p16, None) == lrcc.ERR_ARG
    assert L.lrcc_gather_probe(p16, p16, 4, p16, 0, p16, None) == lrcc.ERR_ARG
    assert L.lrcc_gather_probe(None, p16, 4, p16, 10, p16, None) == lrcc.ERR_ARG


def test_plan_table_roundtrip(lib):
    before = lrcc.get_plan(lrcc.KIND_LR, 1 << 20)
    lrcc.set_plan(lrcc.KIND_LR, 20, 20, rs_spacing0=64)
    assert lrcc.get_plan(lrcc.KIND_LR, 1 << 20)["rs_spacing0"] == 64
    assert lrcc.get_plan(lrcc.KIND_LR, 1 << 21)["rs_spacing0"] == before["rs_spacing0"]
    lrcc.set_plan(lrcc.KIND_LR, 20, 20, rs_spacing0=before["rs_spacing0"])
    with pytest.raises(lrcc.LrccError):
        lrcc.set_plan(lrcc.KIND_LR, 0, 32, rs_small=100000)
    with pytest.raises(lrcc.LrccError):
        lrcc.set_plan(lrcc.KIND_CC, 0, 32, cc_hook=6)
    # hook rule 5 (first pass links the endpoints themselves) is a plan value like the others
    lrcc.set_plan(lrcc.KIND_CC_BATCH, 0, 32, cc_hook=5)
    try:
        assert lrcc.get_plan(lrcc.KIND_CC_BATCH, 1 << 20)["cc_hook"] == 5
    finally:
        lrcc.reset_plans()
    with pytest.raises(lrcc.LrccError):
        lrcc.set_plan(lrcc.KIND_CC, 0, 32, cc_sample=-2)
    # the Shiloach-Vishkin rounds keep one int32 mark per vertex, the other rules active-edge buffers
    L = lrcc.load()
    before = lrcc.get_plan(lrcc.KIND_CC, 1 << 20)["cc_hook"]
    lrcc.set_plan(lrcc.KIND_CC, 20, 20, cc_hook=4)
    try:
        assert L.lrcc_workspace_query(lrcc.KIND_CC, 1 << 20, 1 << 22) == 4 * (1 << 20)
    finally:
        lrcc.set_plan(lrcc.KIND_CC, 20, 20, cc_hook=before)


def test_sparse_graphs_have_their_own_plan_class(lib):
    lrcc.reset_plans()
    # built in: re-linking after a sample pass once a sparse graph's parent array outgrows L2
    assert lrcc.get_plan(lrcc.KIND_CC_SPARSE, 1 << 26)["cc_hook"] == 3
    assert lrcc.get_plan(lrcc.KIND_CC_SPARSE, 1 << 26)["cc_sample"] == 8
    assert lrcc.get_plan(lrcc.KIND_CC, 1 << 26)["cc_hook"] == 1
    assert lrcc.get_plan(lrcc.KIND_CC_SPARSE, 1 << 20) == lrcc.get_plan(lrcc.KIND_CC, 1 << 20)
    # the workspace query takes the class from the edges per vertex
    L = lrcc.load()
    lrcc.set_plan(lrcc.KIND_CC_SPARSE, 20, 20, cc_hook=4)
    try:
        assert L.lrcc_workspace_query(lrcc.KIND_CC, 1 << 20, 3 << 20) == 4 * (1 << 20)   # 3 edges per vertex
        assert L.lrcc_workspace_query(lrcc.KIND_CC, 1 << 20, 1 << 22) != 4 * (1 << 20)   # 4 per vertex: dense
    finally:
        lrcc.reset_plans()
    with pytest.raises(lrcc.LrccError):
        lrcc.set_plan(6, 0, 32, cc_hook=1)


def test_reset_plans_restores_the_builtin_table(lib):
    lrcc.reset_plans()
    before = {k: lrcc.get_plan(k, 1 << 24) for k in (lrcc.KIND_LR, lrcc.KIND_CC, lrcc.KIND_CC_SPARSE, lrcc.KIND_LR_BATCH)}
    lrcc.set_plan(lrcc.KIND_LR, 0, 32, rs_spacing0=128, rs_level0=2, seed=7)
    lrcc.set_plan(lrcc.KIND_CC, 0, 32, cc_hook=4, cc_sample=3)
    lrcc.reset_plans()
    assert {k: lrcc.get_plan(k, 1 << 24) for k in before} == before


def test_workspace_query(lib):
    L = lrcc.load()
    assert L.lrcc_workspace_query(lrcc.KIND_LR, 1000, 0) == 0          # one block, no workspace
    big = L.lrcc_workspace_query(lrcc.KIND_LR, 1 << 28, 0)
    # read-only first level: 8-byte pairs + ~8 bytes of chunked records + small deeper levels
    assert 18 * (1 << 28) <= big < 23 * (1 << 28)
    lrcc.set_plan(lrcc.KIND_LR, 28, 28, rs_level0=1)
    try:
        # in-place first level: 8-byte walk words + small deeper levels
        assert 8 * (1 << 28) <= L.lrcc_workspace_query(lrcc.KIND_LR, 1 << 28, 0) < 9 * (1 << 28)
    finally:
        lrcc.set_plan(lrcc.KIND_LR, 28, 28, rs_level0=2)
    assert L.lrcc_workspace_query(lrcc.KIND_LR_WYLLIE, 1 << 20, 0) == 16 * (1 << 20)
    # weighted ranks: the in-place first level; forests: 37 to 40 bytes per element
    assert 8 * (1 << 24) <= L.lrcc_workspace_query(6, 1 << 24, 0) < 10 * (1 << 24)
    assert 37 * (1 << 24) <= L.lrcc_workspace_query(7, 1 << 24, 0) < 40 * (1 << 24)
    # batched lists of 2^26 elements in all are ranked as one list (the read-only layout)
    assert L.lrcc_workspace_query(lrcc.KIND_LR_BATCH, 1 << 26, 4096) > 18 * (1 << 26)
