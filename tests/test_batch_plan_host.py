"""Host checks of the batched engine's CPU-side parts (csrc/qs_batch_plan.h),
compiled with g++, no GPU: the segment planner's invariants on random
batches, and the superoperators that density-matrix channels and Kraus maps
are lowered to, applied to random Choi vectors and compared with the
oracle's channels (which follow the paper's update rules)."""

import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import qsim_oracle as orc
from paper_2311_01512_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
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
    exe = tmp_path_factory.mktemp("bpc") / "batch_plan_check"
    src = os.path.join(ROOT, "tests", "host", "batch_plan_check.cpp")
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2311_01512_gb300", "csrc"),
                    "-I", os.path.join(ROOT, "include"), "-I", cuda_inc, src, "-o", str(exe)], check=True)

    def run(lines):
        res = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True,
                             timeout=300)
        assert res.returncode == 0, res.stdout + res.stderr
        return res.stdout.splitlines()
    return run


def apply_superop(beta, positions, S):
    """new beta_i = sum_k S[m(i)][k] beta_{base(i) | k deposited on positions}."""
    n = len(positions)
    idx = np.arange(beta.shape[0], dtype=np.int64)
    member = np.zeros_like(idx)
    base = idx.copy()
    for q, p in enumerate(positions):
        member |= ((idx >> p) & 1) << q
        base &= ~(1 << p)
    out = np.zeros_like(beta)
    for k in range(1 << n):
        src = base.copy()
        for q, p in enumerate(positions):
            if (k >> q) & 1:
                src |= 1 << p
        out += S[member, k] * beta[src]
    return out


def numbers(line):
    return np.array([float(v) for v in line.split()])


def test_segment_planner_invariants(harness):
    assert harness(["plan"]) == ["plan ok (0 failures)"]


def test_channel_superops_match_the_oracle(harness):
    rng = np.random.default_rng(5)
    nq = 3
    states, w = wl.random_mixed_state_vectors(nq, 3, rng)
    beta = sum(wi * orc.densmatr_from_pure(v) for wi, v in zip(w, states))
    p, px, py, pz = 0.07, 0.03, 0.02, 0.05
    cases = [
        ("c1 1 0 %r 0" % (1 - 2 * p), [1], lambda b: orc.densmatr_apply_dephasing(b, 1, p)),
        ("c1 %r %r %r 0" % (1 - 2 * p / 3, 2 * p / 3, 1 - 4 * p / 3), [2],
         lambda b: orc.densmatr_apply_depolarising(b, 2, p)),
        ("c1 %r %r %r %r" % (1 - px - py, px + py, 1 - px - py - 2 * pz, px - py), [0],
         lambda b: orc.densmatr_apply_pauli_channel(b, 0, px, py, pz)),
        ("damp %r" % p, [2], lambda b: orc.densmatr_apply_damping(b, 2, p)),
        ("c2 0 %r" % p, [2, 0], lambda b: orc.densmatr_apply_two_qubit_dephasing(b, 2, 0, p)),
        ("c2 1 %r" % p, [0, 2], lambda b: orc.densmatr_apply_two_qubit_depolarising(b, 0, 2, p)),
    ]
    out = harness([c[0] for c in cases])
    for (cmd, targs, ref), line in zip(cases, out):
        v = numbers(line)
        d = int(round(np.sqrt(v.size)))
        positions = list(targs) + [t + nq for t in targs]
        got = apply_superop(beta, positions, v.reshape(d, d))
        assert np.max(np.abs(got - ref(beta))) < 1e-15, cmd


@pytest.mark.parametrize("n", [1, 2])
def test_kraus_superop_matches_the_oracle(harness, n):
    rng = np.random.default_rng(10 + n)
    nq = 4
    states, w = wl.random_mixed_state_vectors(nq, 2, rng)
    beta = sum(wi * orc.densmatr_from_pure(v) for wi, v in zip(w, states))
    kraus = wl.haar_kraus(n, 4, rng)
    flat = np.ascontiguousarray(np.stack(kraus)).view(np.float64).ravel()
    line = harness(["kraus %d %d %s" % (n, len(kraus), " ".join(repr(float(x)) for x in flat))])[0]
    v = numbers(line)
    d = 1 << (2 * n)
    S = (v[0::2] + 1j * v[1::2]).reshape(d, d)
    targs = [3, 1][:n]
    positions = targs + [t + nq for t in targs]
    got = apply_superop(beta, positions, S)
    want = orc.densmatr_apply_kraus(beta, targs, kraus)
    assert np.max(np.abs(got - want)) < 1e-14
