"""Library contexts (lrcc_ctx_*): a stream's workspace reserved ahead of the
calls, counted, and freed with the context."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import gen
import paper_1002_4482_gb300 as lrcc

pytestmark = pytest.mark.gpu


def test_reserve_count_and_destroy():
    dev = torch.device("cuda", 0)
    n = 1 << 22
    succ, head, perm = gen.list_random(n, 71, with_perm=True)
    s = torch.cuda.Stream(dev)
    with torch.cuda.stream(s):
        sd = torch.from_numpy(succ).to(dev)
        out = torch.empty_like(sd)
    s.synchronize()
    before = lrcc.workspace_bytes()
    need = lrcc.workspace_query(lrcc.KIND_LR, n)
    with lrcc.Context(0) as ctx:
        assert ctx.bytes() == 0
        ctx.reserve(s, need)
        held = ctx.bytes()
        assert held >= need
        assert lrcc.workspace_bytes() - before == held
        for _ in range(2):
            lrcc.lr_rank(sd, head, out=out, stream=s)
            assert ctx.last_status(s) == lrcc.OK
            assert ctx.bytes() == held           # the reservation covered the calls
        r = out.cpu().numpy()
        assert np.array_equal(r[perm], np.arange(n - 1, -1, -1, dtype=np.int32))
    assert lrcc.workspace_bytes() == before      # the context freed what it adopted


def test_context_reports_device_errors_of_its_stream():
    dev = torch.device("cuda", 0)
    succ, head = gen.list_random(20_000, 7)
    succ = succ.copy()
    succ[int(np.flatnonzero(succ == -1)[0])] = head   # the whole list becomes a cycle
    s = torch.cuda.Stream(dev)
    ctx = lrcc.Context(0)
    try:
        ctx.reserve(s, 0)
        with torch.cuda.stream(s):
            sd = torch.from_numpy(succ).to(dev)
            out = torch.empty_like(sd)
        lrcc.lr_rank(sd, head, out=out, stream=s)
        assert ctx.last_status(s) == lrcc.ERR_INVALID_INPUT
        assert ctx.last_status(s) == lrcc.OK     # read and cleared
    finally:
        ctx.close()


def test_bad_device_is_an_argument_error():
    with pytest.raises(lrcc.LrccError):
        lrcc.Context(torch.cuda.device_count())


def test_injected_allocation_failure_is_reported_and_recovers():
    dev = torch.device("cuda", 0)
    succ, head, perm = gen.list_random(1 << 20, 73, with_perm=True)
    s = torch.cuda.Stream(dev)
    with torch.cuda.stream(s):
        sd = torch.from_numpy(succ).to(dev)
        out = torch.empty_like(sd)
    s.synchronize()
    try:
        assert lrcc.debug_fail_allocs(1) == 0
        with pytest.raises(lrcc.LrccError) as e:
            lrcc.lr_rank(sd, head, out=out, stream=s)      # a new stream: its workspace is allocated now
        assert e.value.status == lrcc.ERR_NOMEM
        assert lrcc.debug_fail_allocs(0) == 0              # the one injected failure was used
        lrcc.lr_rank(sd, head, out=out, stream=s)
        assert lrcc.last_status(s) == lrcc.OK
        assert np.array_equal(out.cpu().numpy()[perm], np.arange((1 << 20) - 1, -1, -1, dtype=np.int32))
    finally:
        lrcc.debug_fail_allocs(0)
        lrcc.release(s)
