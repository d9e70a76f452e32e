"""Host check of the integer slicing behind the complex128 tensor-core kernel
(paper_2311_01512_gb300/csrc/qs_slices.cuh): exact digits, exact FP32 levels,
exact recombination, dot-product error bound.  Compiled with g++; CPU only."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_integer_slices(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = tmp_path / "slices_check"
    src = os.path.join(ROOT, "tests", "host", "slices_check.cpp")
    inc = os.path.join(ROOT, "paper_2311_01512_gb300", "csrc")
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", inc, src, "-o", str(exe)], check=True)
    res = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stdout + res.stderr
    assert "ok (0 failures)" in res.stdout
