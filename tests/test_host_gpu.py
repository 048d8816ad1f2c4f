"""Host-buffer entry points (lr_rank_host, cc_label_host): the same results as the
device forms and the oracle, bit-exact, from pinned and pageable host memory, with
calls queued on several streams at once."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1002_4482_gb300 as lrcc

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.mark.parametrize("pinned", [True, False], ids=["pinned", "pageable"])
@pytest.mark.parametrize("n", [1, 5, 8193, 300_007])
def test_lr_rank_host_matches_oracle(pinned, n):
    succ, head = gen.list_random(n, 31)
    t = torch.from_numpy(succ)
    if pinned:
        t = t.pin_memory()
    out = torch.empty(n, dtype=torch.int32, pin_memory=pinned)
    rank = lrcc.lr_rank_host(t, head, out=out)
    lrcc.check()
    assert np.array_equal(rank.numpy(), oracle.lr_rank(succ, head))


@pytest.mark.parametrize("pinned", [True, False], ids=["pinned", "pageable"])
def test_cc_label_host_matches_oracle(pinned):
    n = 50_000
    src, dst = gen.er(n, 60_000, 32)
    a, b = torch.from_numpy(src), torch.from_numpy(dst)
    if pinned:
        a, b = a.pin_memory(), b.pin_memory()
    lab = lrcc.cc_label_host(a, b, n)
    lrcc.check()
    assert np.array_equal(lab.numpy(), oracle.cc_uf(src, dst, n))
    # no edges: every vertex alone
    e = torch.empty(0, dtype=torch.int32)
    assert np.array_equal(lrcc.cc_label_host(e, e, 7).numpy(), np.arange(7))


def test_queued_calls_on_alternating_streams():
    # steps alternate between two streams per call, as a pipelined caller would
    # queue them; every output must equal the oracle once its stream is done
    n = 200_003
    lists = [gen.list_random(n, 40 + k) for k in range(4)]
    graphs = [gen.er(60_000, 90_000, 50 + k) for k in range(4)]
    streams = [torch.cuda.Stream(DEV) for _ in range(4)]
    ins, outs = [], []
    for k in range(4):
        succ = torch.from_numpy(lists[k][0]).pin_memory()
        src, dst = (torch.from_numpy(x).pin_memory() for x in graphs[k])
        r = lrcc.lr_rank_host(succ, lists[k][1], stream=streams[k % 2], sync=False)
        lab = lrcc.cc_label_host(src, dst, 60_000, stream=streams[2 + k % 2], sync=False)
        ins.append((succ, src, dst))
        outs.append((r, lab))
    for s in streams:
        s.synchronize()
        assert lrcc.last_status(s) == lrcc.OK
    for k in range(4):
        assert np.array_equal(outs[k][0].numpy(), oracle.lr_rank(*lists[k]))
        assert np.array_equal(outs[k][1].numpy(), oracle.cc_uf(graphs[k][0], graphs[k][1], 60_000))


def test_host_forms_reject_device_tensors_and_report_bad_lists():
    succ, head = gen.list_random(1000, 3)
    with pytest.raises(TypeError):
        lrcc.lr_rank_host(torch.from_numpy(succ).to(DEV), head)
    bad = succ.copy()
    tail = int(np.flatnonzero(bad == -1)[0])
    bad[tail] = head                                   # a cycle
    lrcc.lr_rank_host(torch.from_numpy(bad), head)
    assert lrcc.last_status() == lrcc.ERR_INVALID_INPUT
    with pytest.raises(lrcc.LrccError):
        lrcc.lr_rank_host(torch.from_numpy(succ), 1000)   # head out of range
