"""The allocation-free expectation value (qs_expec_pauli_sum_noalloc) agrees
with the handle-based qs_expec_pauli_sum.

Some callers cannot let a library allocate GPU memory: cudaMalloc/cudaFree
synchronise the device, and some host programs give all device memory to their
own pool.  The allocation-free entry point keeps its scratch in a fixed array
inside the library, shared by every call, so this test calls it twice in a row
with different inputs (a stale term list or partial sum would show) and on
both a statevector and a density matrix.  The file name makes pytest collect
it last.
"""

import numpy as np
import pytest

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
        for call in range(2):
            num_terms = (37, 256)[call]            # second call: the most terms allowed
            paulis, coeffs = wl.random_pauli_sum(n, num_terms, rng)
            want = qs.qs_expec_pauli_sum(state.handle, paulis, coeffs)
            got = qs.qs_expec_pauli_sum_noalloc(state.tensor.data_ptr(), n, is_dm, prec, paulis, coeffs,
                                                state.stream.cuda_stream)
            assert abs(got - want) <= tol, (call, got, want)


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
