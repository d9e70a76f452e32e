"""Host check of the statevector expectation's tile order (qs_internal.h),
compiled with g++, no GPU: the virtual-position map is a bijection and every
term pairs tiles within one block of consecutive positions."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_tile_order(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    cuda_inc = None
    for cand in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "include", "cuda_runtime.h")):
            cuda_inc = os.path.join(cand, "include")
            break
    if cuda_inc is None:
        pytest.skip("CUDA headers not available")
    exe = tmp_path / "tile_order_check"
    src = os.path.join(ROOT, "tests", "host", "tile_order_check.cpp")
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2311_01512_gb300", "csrc"),
                    "-I", os.path.join(ROOT, "include"), "-I", cuda_inc, src, "-o", str(exe)], check=True)
    res = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stdout + res.stderr
    assert "ok (0 failures)" in res.stdout
