"""The multi-threaded CPU baseline ranks correctly (against the oracle); no GPU."""
from __future__ import annotations

import numpy as np
import pytest

import cpu_baseline
import gen
import oracle


@pytest.mark.parametrize("n", [1, 2, 3, 63, 64, 65, 1000, 100_003])
@pytest.mark.parametrize("threads", [1, 3, 8])
def test_cpu_baseline_matches_oracle(n, threads):
    succ, head = gen.list_random(n, 90 + n % 7)
    for spacing in (1, 4, 64):
        assert np.array_equal(cpu_baseline.lr_rank(succ, head, threads, spacing), oracle.lr_rank(succ, head))


def test_cpu_baseline_rejects_invalid_lists():
    with pytest.raises(ValueError):
        cpu_baseline.lr_rank(np.array([1, 0], np.int32), 0)          # cycle
    with pytest.raises(ValueError):
        cpu_baseline.lr_rank(np.array([1, -1, -1], np.int32), 0)     # two lists
