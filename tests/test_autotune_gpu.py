"""The autotuner only installs plans whose results it has checked, and the
library gives the same exact results under the tuned plans."""
from __future__ import annotations

import json

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1002_4482_gb300 as lrcc
from paper_1002_4482_gb300 import autotune

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def test_quick_tune_installs_checked_plans(tmp_path):
    try:
        res = autotune.tune(quick=True, list_classes=(14, 18), graph_classes=(14,), batch_log2=6,
                            log=lambda *a: None)
        path = tmp_path / "plans.json"
        path.write_text(json.dumps(res))
        assert autotune.load(str(path))
        assert lrcc.get_plan(lrcc.KIND_LR, 1 << 18)["rs_spacing0"] == res["lists"]["18"]["plan"]["rs_spacing0"]
        assert lrcc.get_plan(lrcc.KIND_CC_SPARSE, 1 << 14)["cc_hook"] == res["sparse_graphs"]["14"]["plan"]["cc_hook"]
        # results under the tuned plans are still exact
        succ, head = gen.list_random(200_000, 5)
        r = lrcc.lr_rank(torch.from_numpy(succ).to(DEV), head).cpu().numpy()
        assert np.array_equal(r, oracle.lr_rank(succ, head))
        src, dst = gen.er(20_000, 60_000, 6)
        lab = lrcc.cc_label(torch.from_numpy(src).to(DEV), torch.from_numpy(dst).to(DEV), 20_000).cpu().numpy()
        assert np.array_equal(lab, oracle.cc_uf(src, dst, 20_000))
    finally:
        _restore_builtin_plans()


def _restore_builtin_plans():
    lrcc.reset_plans()
