"""bench.py's own arm on the GPU, small workload: one JSON line with the keys
the benchmark contract asks for (roofline, CPU baseline, end-to-end leg,
clocks, launch count) and the rows of the kernel table."""
from __future__ import annotations

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu


def test_small_workload_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--workload", "small", "--steps", "3",
                        "--warmup", "3", "--no-batched", "--no-serve", "--no-families", "--no-sweep"],
                       capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "clocks", "e2e", "gpu_launches", "roofline",
                "cpu_baseline"):
        assert key in d, key
    assert d["value"] > 0 and d["n_gpus"] == 1 and d["steps"] == 3 and d["gpu_launches"] > 0
    assert d["config"]["workload"] == "lr_random_2p20+cc_er_2p20_2p22"
    e2e = d["e2e"]
    assert e2e["value"] > 0 and e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] > 0
    roof = d["roofline"]
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in roof, key
    assert 0 < roof["frac"] < 2
    assert {k["kernel"].split(" ")[0] for k in roof["other_kernels"]} >= {"cc_hook"}
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    g = d["cc"]["gather_ceiling"]
    assert g["probe_ms_per_pass"] > 0 and g["full_pass_ms"] > 0
    assert d["step_ms"]["two_streams_ms"] > 0
