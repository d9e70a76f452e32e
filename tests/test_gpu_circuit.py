"""Planned circuits with gate fusion (qs_circuit_*) against the CPU oracle.

Fusion regroups the same unitary operations into dense blocks composed in
FP64, so the planned result must equal the gate-by-gate oracle result within
the same tolerances as single operations: complex128 1e-12 per 1000 gates,
complex64 (tensor cores, 3xTF32) FP32-level."""

import numpy as np
import pytest

from oracle import qsim_oracle as orc
from paper_2311_01512_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    from paper_2311_01512_gb300 import qs as mod
    return mod


def run_plan(qs, nq, density, prec, init, ops, kind, width):
    circ = qs.Circuit(nq, ops)
    stats = circ.plan(kind, width)
    st = qs.State(nq, density=density, prec=prec)
    st.set_amps(init)
    circ.apply(st.handle)
    qs.qs_synchronize(st.handle)
    out = st.get_amps().astype(np.complex128)
    st.close()
    circ.close()
    return out, stats


@pytest.mark.parametrize("width", [2, 4, 5, 6])
def test_statevector_circuit_fused_c128(qs, width):
    rng = wl.rng_for("fuse-sv12-%d" % width)
    nq = 12
    psi = wl.random_statevector(nq, rng)
    ops = wl.statevector_circuit(nq, 160, rng, max_targs=3, max_ctrls=2)
    want = orc.run_ops(psi, ops, is_density=False)
    got, stats = run_plan(qs, nq, False, 1, psi, ops, qs.QS_PLAN_GREEDY, width)
    assert stats["gates"] == 160 and stats["blocks"] < 160 and stats["fused"] > 0
    assert float(np.max(np.abs(got - want))) <= 0.3e-12


@pytest.mark.parametrize("width", [5, 6])
def test_unitary_circuit_fused_c64_tensor_cores(qs, width):
    """Width 6 puts the 6-target blocks on the bf16-slice kernel."""
    rng = wl.rng_for("fuse-c64")
    nq = 14
    psi = wl.random_statevector(nq, rng)
    ops = wl.unitary_circuit(nq, 200, rng)
    want = orc.run_ops(psi, ops, is_density=False)
    got_fused, stats = run_plan(qs, nq, False, 0, psi.astype(np.complex64), ops, qs.QS_PLAN_GREEDY, width)
    got_plain, _ = run_plan(qs, nq, False, 0, psi.astype(np.complex64), ops, qs.QS_PLAN_NONE, 1)
    scale = float(np.max(np.abs(want)))
    err_f = float(np.max(np.abs(got_fused - want)))
    err_p = float(np.max(np.abs(got_plain - want)))
    assert stats["blocks"] < 120
    # 200 gates in FP32-level arithmetic, as fused blocks or gate by gate
    assert err_f <= 200 * scale * 2.0 ** -22, (err_f, err_p)
    fid = abs(np.vdot(want, got_fused)) ** 2 / (np.vdot(want, want).real * np.vdot(got_fused, got_fused).real)
    assert 1.0 - fid <= 1e-6


def test_density_circuit_fused_c128(qs):
    rng = wl.rng_for("fuse-dm5")
    nq = 5
    states, w = wl.random_mixed_state_vectors(nq, 3, rng)
    beta = sum(wi * orc.densmatr_from_pure(s) for wi, s in zip(w, states))
    ops = wl.unitary_circuit(nq, 60, rng)
    want = orc.run_ops(beta, ops, is_density=True)
    got, stats = run_plan(qs, nq, True, 1, beta, ops, qs.QS_PLAN_GREEDY, 3)
    assert stats["fused"] > 0
    assert float(np.max(np.abs(got - want))) <= 1e-13


def test_plan_validation(qs):
    circ = qs.Circuit(4)
    with pytest.raises(qs.QSError):
        circ.plan(qs.QS_PLAN_GREEDY, 7)          # wider than a dense gate allows
    with pytest.raises(qs.QSError):
        circ.add({"op": "unitary", "ctrls": [1], "targs": [1], "mat": np.eye(2)})
    circ.add({"op": "unitary", "ctrls": [], "targs": [0], "mat": np.eye(2)})
    st = qs.State(5)
    with pytest.raises(qs.QSError):
        circ.apply(st.handle)                    # qubit count differs


def test_fused_c64_matches_per_gate_c128_at_22_qubits(qs):
    """A size-independent property at a size beyond the oracle's comfort: the
    cost-planned tensor-core complex64 result has 1 - F <= 1e-6 against the
    per-gate complex128 result (itself oracle-checked at small sizes)."""
    import torch
    from paper_2311_01512_gb300 import costmodel
    nq = 22
    rng = wl.rng_for("fuse-22")
    psi = wl.random_statevector(nq, rng)
    ops = wl.unitary_circuit(nq, 300, rng)
    ref, _ = run_plan(qs, nq, False, 1, psi, ops, qs.QS_PLAN_NONE, 1)
    for plan, width in (("greedy", 5), ("greedy", 6), ("cost", 5), ("cost", 6)):
        circ = qs.Circuit(nq, ops)
        st = qs.State(nq, prec=0)
        st.set_amps(psi.astype(np.complex64))
        if plan == "greedy":
            circ.plan(qs.QS_PLAN_GREEDY, width)
        else:
            model, _ = costmodel.load()
            circ.plan_cost(model, st.handle, max_block_qubits=width, window=24)
        circ.apply(st.handle)
        qs.qs_synchronize(st.handle)
        got = st.get_amps().astype(np.complex128)
        fid = abs(np.vdot(ref, got)) ** 2 / (np.vdot(ref, ref).real * np.vdot(got, got).real)
        assert 1.0 - fid <= 1e-6, (plan, width, 1.0 - fid)


@pytest.mark.parametrize("prec", [1, 0])
def test_relabelled_circuit_matches_oracle(qs, prec):
    """Lazy relabelling with its SWAP price set so low that every tensor-core
    block with a qubit among the 5 lowest positions gets SWAPs: the circuit's
    result must still equal the gate-by-gate oracle (the layout is restored at
    the end), and replanning clears the relabelling."""
    from paper_2311_01512_gb300 import costmodel
    rng = wl.rng_for("relabel-%d" % prec)
    nq = 13
    psi = wl.random_statevector(nq, rng)
    ops = wl.unitary_circuit(nq, 150, rng)
    want = orc.run_ops(psi, ops, is_density=False)
    dtype = np.complex128 if prec == 1 else np.complex64
    st = qs.State(nq, density=False, prec=prec)
    st.set_amps(psi.astype(dtype))
    model, _ = costmodel.load()
    circ = qs.Circuit(nq, ops)
    circ.plan_cost(model, st.handle, max_block_qubits=5 if prec == 1 else 6, window=16)
    nswaps = circ.plan_relabel(model, st.handle, low_qubits=5, swap_passes=-1e30)
    assert nswaps > 0
    circ.apply(st.handle)
    qs.qs_synchronize(st.handle)
    got = st.get_amps().astype(np.complex128)
    # complex64: 150 gates in FP32-level arithmetic, as in the fused complex64 test
    tol = 2e-14 if prec == 1 else 150 * 2.0 ** -22 * float(np.max(np.abs(want)))
    assert float(np.max(np.abs(got - want))) <= tol
    assert circ.plan_relabel(model, st.handle, low_qubits=0) == 0
    circ.plan(qs.QS_PLAN_GREEDY, 4)
    assert circ.plan_relabel(model, st.handle, low_qubits=5, swap_passes=1e30) == 0
    circ.close()
    model.close()
    st.close()
