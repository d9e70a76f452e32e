"""Host check of the one-qubit superoperator that the library forms on the
host for one-pass Kraus maps and one-qubit density-matrix unitaries
(paper_2311_01512_gb300/csrc/qs_superop1.h, driven by
tests/host/superop1_check.cpp): against the oracle's superoperator
sum_m conj(K_m) (x) K_m (Sec. "Kraus map"), and, applied as a two-target gate
on (t, t + N) of a Choi vector, against the oracle's Kraus map and unitary on
a density matrix.  CPU only."""

import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import qsim_oracle as orc
from paper_2311_01512_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = tmp_path_factory.mktemp("superop1") / "superop1_check"
    src = os.path.join(ROOT, "tests", "host", "superop1_check.cpp")
    inc = os.path.join(ROOT, "paper_2311_01512_gb300", "csrc")
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", inc, src, "-o", str(out)], check=True)
    return str(out)


def run(exe, kraus_sets):
    lines = []
    for ks in kraus_sets:
        flat = np.concatenate([np.stack([k.real, k.imag], -1).reshape(-1) for k in ks])
        lines.append(" ".join([str(len(ks))] + [float(v).hex() for v in flat]))
    res = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=60)
    assert res.returncode == 0, res.stderr
    out = []
    for line in res.stdout.split("\n"):
        if line.strip():
            v = np.array([float.fromhex(x) for x in line.split()])
            out.append((v[0::2] + 1j * v[1::2]).reshape(4, 4))
    assert len(out) == len(kraus_sets)
    return out


def test_superop1_matches_oracle(exe):
    rng = np.random.default_rng(2311)
    sets = [wl.haar_kraus(1, m, rng) for m in (1, 2, 3, 4) for _ in range(50)]
    sets += [[wl.haar_unitary(2, rng)] for _ in range(50)]
    # non-unitary, unnormalised operators with entries over many binades
    sets += [[rng.standard_normal((2, 2)) * 10.0 ** rng.uniform(-8, 3, (2, 2)) + 1j * rng.standard_normal((2, 2))
              for _ in range(3)] for _ in range(20)]
    for ks, got in zip(sets, run(exe, sets)):
        want = orc.superoperator(ks)
        scale = max(float(np.max(np.abs(want))), 1e-300)
        assert float(np.max(np.abs(got - want))) <= 4e-16 * scale * len(ks)


def test_superop1_as_two_target_pass_on_choi_vector(exe):
    """The pass the library makes: the superoperator on (t, t + N) of the Choi
    vector, matrix bit 0 on t, bit 1 on t + N."""
    rng = np.random.default_rng(2312)
    nq = 3
    pure = [wl.random_statevector(nq, rng) for _ in range(2)]
    rho = 0.6 * orc.densmatr_from_pure(pure[0]) + 0.4 * orc.densmatr_from_pure(pure[1])
    for t in range(nq):
        kraus = wl.haar_kraus(1, 3, rng)
        u = wl.haar_unitary(2, rng)
        s_k, s_u = run(exe, [kraus, [u]])
        got = orc.apply_ctrl_multi_target(rho, [], [t, t + nq], s_k)
        assert np.allclose(got, orc.densmatr_apply_kraus(rho, [t], kraus), atol=1e-15)
        got = orc.apply_ctrl_multi_target(rho, [], [t, t + nq], s_u)
        assert np.allclose(got, orc.densmatr_apply_ctrl_multi_target(rho, [], [t], u), atol=1e-15)
