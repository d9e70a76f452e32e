"""Failure handling, with every failure made on the host (no GPU fault, trap
or hang): library allocations made to fail by qs_test_fail_allocations must
give QS_ERR_OOM, leave no handle and leak nothing; a handle's device error
word set from the host (as a tensor-core kernel sets it when a bounded wait
runs out) must come back once as QS_ERR_TIMEOUT from qs_synchronize, with
the state still usable.  The paper has no counterpart: it assumes reliable
MPI and memory."""

import ctypes

import numpy as np
import pytest

from oracle import qsim_oracle as orc
from paper_2311_01512_gb300 import workloads as wl

QS_ERR_OOM = 7


@pytest.fixture(scope="module")
def qs():
    from paper_2311_01512_gb300 import qs as mod
    return mod


def create_raw(qs, nq, dptr):
    h = ctypes.c_void_p()
    st = qs._lib.qs_create_statevector(nq, qs.QS_C128, ctypes.c_void_p(dptr), None, ctypes.byref(h))
    return st, h


def test_injected_allocation_failure_on_the_host(qs):
    """The first allocation of a new handle fails before CUDA is called, so
    this runs without a GPU: QS_ERR_OOM and no handle."""
    try:
        qs.qs_test_fail_allocations(0, 1)
        st, h = create_raw(qs, 10, 256 * 4096)     # aligned, never dereferenced
        assert st == QS_ERR_OOM
        assert not h.value
    finally:
        qs.qs_test_fail_allocations(0, 0)
    with pytest.raises(qs.QSError) as ei:
        qs.qs_test_fail_allocations(-1, 1)
    assert "QS_ERR_ARG" in str(ei.value)


@pytest.mark.gpu
def test_every_handle_allocation_failure_frees_the_others(qs):
    """A handle takes four allocations (scratch, device ring, pinned result,
    pinned ring); failing each in turn gives QS_ERR_OOM and leaves device
    memory as it was; afterwards a handle is created and works."""
    import torch
    nq = 8
    psi = torch.zeros(1 << nq, dtype=torch.complex128, device="cuda")
    st, h = create_raw(qs, nq, psi.data_ptr())     # one full create and destroy first
    assert st == 0
    assert qs._lib.qs_destroy(h) == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    try:
        for skip in range(4):
            qs.qs_test_fail_allocations(skip, 1)
            st, h = create_raw(qs, nq, psi.data_ptr())
            assert st == QS_ERR_OOM, skip
            assert not h.value
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info()[0] == free0, skip
    finally:
        qs.qs_test_fail_allocations(0, 0)
    s = qs.State(nq, density=False, prec=qs.QS_C128)
    vec = wl.random_statevector(nq, np.random.default_rng(5))
    s.set_amps(vec)
    qs.qs_apply_ctrl_multi_target(s.handle, [], [3], wl.haar_unitary(2, np.random.default_rng(6)))
    assert abs(qs.qs_calc_norm_or_trace(s.handle) - 1.0) < 1e-14
    s.close()


@pytest.mark.gpu
def test_circuit_and_program_allocation_failures(qs):
    """A fused plan whose block matrices cannot be allocated, and a recorded
    program whose matrix arena cannot be allocated, both give QS_ERR_OOM;
    with the injection off the same calls succeed and agree with the oracle."""
    rng = wl.rng_for("alloc-failure")
    nq = 9
    ops = wl.unitary_circuit(nq, 40, rng)
    psi = wl.random_statevector(nq, rng)
    circ = qs.Circuit(nq, ops)
    try:
        qs.qs_test_fail_allocations(0, 1)
        with pytest.raises(qs.QSError) as ei:
            circ.plan(qs.QS_PLAN_GREEDY, 4)
        assert "QS_ERR_OOM" in str(ei.value)
    finally:
        qs.qs_test_fail_allocations(0, 0)
    circ.plan(qs.QS_PLAN_GREEDY, 4)
    import torch
    st = qs.State(nq, density=False, prec=qs.QS_C128, stream=torch.cuda.Stream())
    st.set_amps(psi)
    circ.apply(st.handle)
    want = orc.run_ops(psi, ops, is_density=False)
    assert float(np.max(np.abs(st.get_amps() - want))) < 1e-13
    # recorded program: its matrix arena is allocated when recording begins
    try:
        qs.qs_test_fail_allocations(0, 1)
        with pytest.raises(qs.QSError) as ei:
            qs.qs_record_begin(st.handle)
        assert "QS_ERR_OOM" in str(ei.value)
    finally:
        qs.qs_test_fail_allocations(0, 0)
    st.set_amps(psi)
    qs.qs_record_begin(st.handle)
    for op in ops:
        qs.apply_op(st.handle, op)
    prog = qs.qs_record_end(st.handle)
    qs.qs_program_run(prog)
    qs.qs_synchronize(st.handle)
    assert float(np.max(np.abs(st.get_amps() - want))) < 1e-13
    qs.qs_program_destroy(prog)
    circ.close()
    st.close()


@pytest.mark.gpu
def test_error_word_reported_once_as_timeout(qs):
    nq = 10
    rng = np.random.default_rng(77)
    psi = wl.random_statevector(nq, rng)
    st = qs.State(nq, density=False, prec=qs.QS_C128)
    st.set_amps(psi)
    qs.qs_synchronize(st.handle)
    qs.qs_test_set_error_word(st.handle)
    with pytest.raises(qs.QSError) as ei:
        qs.qs_synchronize(st.handle)
    assert "QS_ERR_TIMEOUT" in str(ei.value)
    qs.qs_synchronize(st.handle)             # reported once, then cleared
    # the handle keeps working: a tensor-core gate and the oracle agree
    u = wl.haar_unitary(8, rng)
    qs.qs_apply_ctrl_multi_target(st.handle, [], [1, 4, 7], u)
    qs.qs_synchronize(st.handle)
    want = orc.apply_ctrl_multi_target(psi, [], [1, 4, 7], u)
    assert float(np.max(np.abs(st.get_amps() - want))) < 1e-14
    st.close()


@pytest.mark.gpu
def test_device_wait_runs_out_and_reports(qs):
    """A wait on a barrier that nothing arrives at gives up after its bounded
    number of polls on the GPU and sets the error word; qs_synchronize reports
    QS_ERR_TIMEOUT once and the handle keeps working."""
    nq = 8
    rng = np.random.default_rng(88)
    psi = wl.random_statevector(nq, rng)
    st = qs.State(nq, density=False, prec=qs.QS_C128)
    st.set_amps(psi)
    qs.qs_synchronize(st.handle)
    qs.qs_test_bounded_wait(st.handle, 4096)
    with pytest.raises(qs.QSError) as ei:
        qs.qs_synchronize(st.handle)
    assert "QS_ERR_TIMEOUT" in str(ei.value)
    qs.qs_synchronize(st.handle)
    with pytest.raises(qs.QSError):
        qs.qs_test_bounded_wait(st.handle, (1 << 20) + 1)
    u = wl.haar_unitary(2, rng)
    qs.qs_apply_ctrl_multi_target(st.handle, [], [5], u)
    want = orc.apply_ctrl_multi_target(psi, [], [5], u)
    assert float(np.max(np.abs(st.get_amps() - want))) < 1e-14
    st.close()
