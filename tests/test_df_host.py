"""Host check of the double-float split / join / dot-product logic that the
complex128 kernels run (paper_2311_01512_gb300/csrc/qs_df.cuh): compiled for
the CPU with g++ and run on random and edge-case inputs.  CPU only."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_df_split_join_dot(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = tmp_path / "df_check"
    src = os.path.join(ROOT, "tests", "host", "df_check.cpp")
    inc = os.path.join(ROOT, "paper_2311_01512_gb300", "csrc")
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", inc, src, "-o", str(exe)], check=True)
    res = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stdout + res.stderr
    assert "ok (0 failures)" in res.stdout
