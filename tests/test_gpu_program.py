"""Recorded programs (qs_record_begin / qs_record_end / qs_program_run): the
operations applied between begin and end are captured once, change nothing
while recording, and each replay equals applying them again (CPU oracle).
Covered: a 6-qubit density matrix with every channel kind, Kraus maps,
gadgets, SWAP and diagonals; statevectors with dense gates on up to 5
targets and controls, in both precisions; calls refused while recording."""

import numpy as np
import pytest

from oracle import qsim_oracle as orc
from paper_2311_01512_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    from paper_2311_01512_gb300 import qs as mod
    return mod


def test_program_density_matrix(qs):
    import torch
    rng = wl.rng_for("program-dm6")
    nq = 6
    stream = torch.cuda.Stream()
    states, w = wl.random_mixed_state_vectors(nq, 4, rng)
    rho0 = sum(wi * orc.densmatr_from_pure(s) for wi, s in zip(w, states))
    dm = qs.State(nq, density=True, prec=qs.QS_C128, stream=stream)
    dm.set_amps(rho0)
    ops = wl.small_densmatr_circuit(nq, 120, rng)
    ops += [
        {"op": "dephasing", "targs": [3], "p": 0.07},
        {"op": "dephasing2", "targs": [0, 5], "p": 0.04},
        {"op": "depolarising2", "targs": [4, 1], "p": 0.05},
        {"op": "pauli_channel", "targs": [2], "probs": (0.02, 0.03, 0.01)},
        {"op": "swap", "targs": [1, 4]},
        {"op": "diagonal", "targs": [5, 0], "diag": np.exp(1j * rng.uniform(0, 2 * np.pi, 4))},
        {"op": "unitary", "ctrls": [], "targs": [2, 3], "mat": wl.haar_unitary(4, rng)},
    ]
    qs.qs_record_begin(dm.handle)
    for op in ops:
        qs.apply_op(dm.handle, op)
    with pytest.raises(qs.QSError):
        qs.qs_calc_norm_or_trace(dm.handle)
    with pytest.raises(qs.QSError):
        qs.qs_synchronize(dm.handle)
    with pytest.raises(qs.QSError):
        qs.qs_record_begin(dm.handle)            # one recording at a time
    prog = qs.qs_record_end(dm.handle)
    assert np.array_equal(dm.get_amps(), rho0)   # recording applied nothing
    qs.qs_program_run(prog)
    qs.qs_program_run(prog)
    want = orc.run_ops(orc.run_ops(rho0, ops, True), ops, True)
    err = float(np.max(np.abs(dm.get_amps() - want)))
    assert err <= 1e-12, err
    qs.qs_program_destroy(prog)
    assert abs(qs.qs_calc_norm_or_trace(dm.handle) - 1.0) < 1e-12


@pytest.mark.parametrize("prec", [1, 0])
def test_program_statevector(qs, prec):
    import torch
    rng = wl.rng_for("program-sv-%d" % prec)
    nq = 12
    stream = torch.cuda.Stream()
    psi = wl.random_statevector(nq, rng)
    st = qs.State(nq, prec=prec, stream=stream)
    st.set_amps(psi)
    ops = wl.statevector_circuit(nq, 80, rng)
    qs.qs_record_begin(st.handle)
    for op in ops:
        qs.apply_op(st.handle, op)
    prog = qs.qs_record_end(st.handle)
    for _ in range(2):
        qs.qs_program_run(prog)
    want = orc.run_ops(orc.run_ops(psi, ops, False), ops, False)
    got = st.get_amps().astype(np.complex128)
    if prec == 1:
        err = float(np.max(np.abs(got - want)))
        assert err <= 1e-12, err
    else:
        fid = abs(np.vdot(want, got)) ** 2 / (np.vdot(got, got).real * np.vdot(want, want).real)
        assert 1.0 - fid <= 1e-6, 1.0 - fid
    qs.qs_program_destroy(prog)


def test_program_refusals(qs):
    import torch
    st = qs.State(4, prec=qs.QS_C128, stream=torch.cuda.Stream())
    with pytest.raises(qs.QSError):
        qs.qs_record_end(st.handle)               # not recording
    qs.qs_record_begin(st.handle)
    with pytest.raises(qs.QSError):
        qs.qs_get_amps(st.handle, np.empty(16, dtype=np.complex128))
    with pytest.raises(qs.QSError):
        qs.qs_destroy(st.handle)
    prog = qs.qs_record_end(st.handle)            # an empty program
    qs.qs_program_run(prog)
    qs.qs_program_destroy(prog)
    legacy = qs.State(4, prec=qs.QS_C128, stream=torch.cuda.default_stream())
    if legacy.stream.cuda_stream == 0:
        with pytest.raises(qs.QSError):
            qs.qs_record_begin(legacy.handle)     # the legacy default stream cannot be captured
