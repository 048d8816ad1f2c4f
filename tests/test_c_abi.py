"""The boundary from plain C: `tests/c_abi/abi_check.c` includes only
`include/lrcc.h` and the CUDA runtime, links liblrcc.so, and checks lr_rank,
lr_rank_wyllie, cc_label and lr_rank_host against closed forms, a context
(create, reserve a stream's workspace, rank on it, count, destroy), plus the
error paths. Compiling and linking it needs no GPU; running it does."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

from paper_1002_4482_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _compile(out: str) -> None:
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    _build.build()
    libdir = os.path.dirname(_build.OUT)
    cmd = [gcc, "-std=c11", "-O2", "-Wall", "-Wextra", "-Werror",
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include"),
           os.path.join(ROOT, "tests", "c_abi", "abi_check.c"),
           "-L", libdir, "-llrcc", "-L", os.path.join(CUDA, "lib64"), "-lcudart",
           f"-Wl,-rpath,{libdir}:{os.path.join(CUDA, 'lib64')}", "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_header_compiles_and_links_from_c(tmp_path):
    _compile(str(tmp_path / "abi_check"))


@pytest.mark.gpu
@pytest.mark.parametrize("n", [2, 16385, 300007, 1 << 22])
def test_c_program_ranks_and_labels(tmp_path, n):
    exe = str(tmp_path / "abi_check")
    _compile(exe)
    r = subprocess.run([exe, str(n)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "abi_check ok" in r.stdout
