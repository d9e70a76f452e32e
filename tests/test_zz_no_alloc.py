"""The allocation-free expectation value (qs_expec_pauli_sum_noalloc) agrees
with the handle-based qs_expec_pauli_sum and with the CPU oracle.

Some callers cannot let a library allocate GPU memory: cudaMalloc/cudaFree
synchronise the device, and some host programs give all device memory to their
own pool.  The allocation-free entry point keeps its scratch in a fixed array
inside the library, shared by every call, so this test calls it twice in a row
with different inputs (a stale term list or partial sum would show) and on
both a statevector and a density matrix.  A 21-qubit statevector gives the
reduction's 1216 blocks several 1024-amplitude tiles each.  The file name
makes pytest collect it last.
"""

import numpy as np
import pytest

from oracle import qsim_oracle as orc
from paper_2311_01512_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    from paper_2311_01512_gb300 import qs as mod
    return mod


@pytest.mark.parametrize("prec", [1, 0])
def test_noalloc_matches_handle_path_twice(qs, prec):
    tol = 1e-12 if prec == 1 else 1e-5
    rng = np.random.default_rng(4242 + prec)
    dtype = np.complex128 if prec == 1 else np.complex64

    nq = 12
    sv = qs.State(nq, density=False, prec=prec)
    sv.set_amps(wl.random_statevector(nq, rng).astype(dtype))
    nd = 5
    dm = qs.State(nd, density=True, prec=prec)
    psis = [wl.random_statevector(nd, rng) for _ in range(2)]
    for m, p in enumerate(psis):
        tmp = qs.State(nd, density=False, prec=prec)
        tmp.set_amps(p.astype(dtype))
        qs.qs_init_pure_densmatr(dm.handle, tmp.handle, 0.5, accumulate=m > 0)
        qs.qs_synchronize(dm.handle)
        tmp.close()

    for state, n, is_dm in ((sv, nq, False), (dm, nd, True)):
        amps = state.get_amps().astype(np.complex128)   # the stored amplitudes, for the oracle
        for call in range(2):
            num_terms = (37, 256)[call]            # second call: the most terms allowed
            paulis, coeffs = wl.random_pauli_sum(n, num_terms, rng)
            want = qs.qs_expec_pauli_sum(state.handle, paulis, coeffs)
            got = qs.qs_expec_pauli_sum_noalloc(state.tensor.data_ptr(), n, is_dm, prec, paulis, coeffs,
                                                state.stream.cuda_stream)
            assert abs(got - want) <= tol, (call, got, want)
            f = orc.expec_pauli_sum_densmatr if is_dm else orc.expec_pauli_sum_statevector
            want_orc = f(amps, paulis, coeffs)
            assert abs(got.real - want_orc.real) <= tol * np.abs(coeffs).sum(), (call, got, want_orc)


@pytest.mark.parametrize("prec", [1, 0])
def test_noalloc_21_qubits_against_oracle(qs, prec):
    """2^21 amplitudes: 2048 tiles of 1024 over the 1216 reduction blocks, so
    blocks take a second tile; two calls in a row with different term lists,
    compared with the handle path and with the oracle."""
    rng = np.random.default_rng(2121 + prec)
    dtype = np.complex128 if prec == 1 else np.complex64
    nq = 21
    psi = wl.random_statevector(nq, rng).astype(dtype)
    sv = qs.State(nq, density=False, prec=prec)
    sv.set_amps(psi)
    tol = 1e-14 if prec == 1 else 1e-5
    for call in range(2):
        paulis, coeffs = wl.random_pauli_sum(nq, (19, 64)[call], rng)
        got = qs.qs_expec_pauli_sum_noalloc(sv.tensor.data_ptr(), nq, False, prec, paulis, coeffs,
                                            sv.stream.cuda_stream)
        want = qs.qs_expec_pauli_sum(sv.handle, paulis, coeffs)
        want_orc = orc.expec_pauli_sum_statevector(psi.astype(np.complex128), paulis, coeffs)
        scale = np.abs(coeffs).sum()
        assert abs(got - want) <= tol * scale, (call, got, want)
        assert abs(got.real - want_orc.real) <= tol * scale, (call, got, want_orc)
    sv.close()


def test_noalloc_rejects_too_many_terms(qs):
    import ctypes
    sv = qs.State(4, density=False)
    qs.qs_init_zero(sv.handle)
    paulis = np.zeros((qs.NOALLOC_MAX_TERMS + 1, 4), dtype=np.int32)
    coeffs = np.ones(qs.NOALLOC_MAX_TERMS + 1)
    with pytest.raises(ValueError, match="at most 256 terms"):
        qs.qs_expec_pauli_sum_noalloc(sv.tensor.data_ptr(), 4, False, 1, paulis, coeffs, sv.stream.cuda_stream)
    out = (ctypes.c_double * 2)()
    status = qs._lib.qs_expec_pauli_sum_noalloc(
        ctypes.c_void_p(sv.tensor.data_ptr()), 4, 0, 1,
        paulis.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), coeffs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        qs.NOALLOC_MAX_TERMS + 1, ctypes.c_void_p(sv.stream.cuda_stream), out)
    assert status == 1      # QS_ERR_ARG
