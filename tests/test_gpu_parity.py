"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Sizes span several shared-memory tiles (a tile is 2^10 amplitudes) and ragged
cases (states with fewer free qubits than a tile, gates with no free qubits
at all).  Integer-valued results (which amplitudes an operation touches) are
checked exactly through the parity of untouched amplitudes.

Tolerances (amplitudes are at most 1 in modulus):
* complex128, block fixed point (the default) and native FP64: 1e-14 absolute
  per operation.  One output of either is within a few units of 2^-53 of the
  largest amplitude it combines (fixed point: 2^-53 |y| + 2^-55 max|x| max|m|
  for K <= 4 terms; 8-slice dense gates (K + 1) 2^-54 of the row and column
  maxima), and so is the oracle's own FP64 result; 1e-14 leaves a factor of
  about 10 over 2^-53 for the K <= 64 terms of a 6-target gate.  Circuits of
  300-500 operations: 2e-14 (errors of successive unitary operations add at
  most, and mostly cancel).
* complex128, double-float (47-bit): 1e-13 per operation, 1e-12 per 1000
  operations.
* complex64: 2e-6 per operation, circuits scaled by the number of operations.
"""

import numpy as np
import pytest

from oracle import qsim_oracle as orc
from paper_2311_01512_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

# precision modes: 1 = complex128 with the default block fixed-point arithmetic,
# 3 = complex128 with double-float, 2 = complex128 with native FP64, 0 = complex64
ATOL = {1: 1e-14, 3: 1e-13, 2: 1e-14, 0: 2e-6}
# scalar results (norm, trace, expectation values) per unit of sum |h| or of
# the trace
STOL = {1: 1e-14, 3: 1e-12, 2: 1e-14, 0: 1e-5}
# circuits of 300-500 operations, max |delta amp|
CTOL = {1: 2e-14, 3: 0.5e-12, 2: 2e-14}


@pytest.fixture(scope="module")
def qs():
    from paper_2311_01512_gb300 import qs as mod
    return mod


def make_state(qs, nq, density, mode):
    st = qs.State(nq, density=density, prec=0 if mode == 0 else 1)
    if mode == 2:
        qs.qs_set_arithmetic(st.handle, qs.QS_ARITH_F64)
    if mode == 3:
        qs.qs_set_arithmetic(st.handle, qs.QS_ARITH_DF)
    return st


def new_sv(qs, nq, prec, psi):
    st = make_state(qs, nq, False, prec)
    st.set_amps(psi)
    return st


def new_dm(qs, nq, prec, beta):
    st = make_state(qs, nq, True, prec)
    st.set_amps(beta)
    return st


def rand_dm(nq, rank, rng):
    states, w = wl.random_mixed_state_vectors(nq, rank, rng)
    return sum(wi * orc.densmatr_from_pure(s) for wi, s in zip(w, states))


def close(got, want, prec, scale=1.0):
    err = float(np.max(np.abs(np.asarray(got, dtype=np.complex128) - want)))
    assert err <= ATOL[prec] * scale, "max |delta amp| = %.3e" % err
    return err


PRECS = [1, 3, 2, 0]


# ---------------------------------------------------------------------------
# statevector gates
# ---------------------------------------------------------------------------

def gate_cases():
    cases = []
    for nq in (10, 13):
        for n in range(1, 7):
            for s in (0, 1, 3):
                cases.append((nq, n, s))
    cases += [(6, 6, 0), (8, 6, 2), (7, 5, 2), (1, 1, 0), (2, 1, 1), (5, 2, 3), (11, 1, 10)]
    return cases


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("nq,n,s", gate_cases())
def test_ctrl_multi_target_gate(qs, prec, nq, n, s):
    rng = np.random.default_rng(1000 * nq + 10 * n + s)
    placements = []
    for _ in range(2):
        qsel = [int(x) for x in rng.choice(nq, n + s, replace=False)]
        placements.append((qsel[:n], qsel[n:]))
    placements.append((list(range(n)), list(range(n, n + s))))                         # lowest qubits
    placements.append((list(range(nq - 1, nq - 1 - n, -1)), list(range(s))))            # highest, reversed
    for targs, ctrls in placements:
        psi = wl.random_statevector(nq, rng)
        mat = rng.standard_normal((1 << n, 1 << n)) + 1j * rng.standard_normal((1 << n, 1 << n))
        mat /= np.sqrt(1 << n)
        st = new_sv(qs, nq, prec, psi)
        qs.qs_apply_ctrl_multi_target(st.handle, ctrls, targs, mat)
        want = orc.apply_ctrl_multi_target(psi, ctrls, targs, mat)
        close(st.get_amps(), want, prec, scale=4)
        st.close()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("nq", [2, 7, 12])
def test_swap(qs, prec, nq):
    rng = np.random.default_rng(700 + nq)
    psi = wl.random_statevector(nq, rng)
    st = new_sv(qs, nq, prec, psi)
    want = psi
    pairs = [(0, nq - 1), (nq - 1, 0)] + [tuple(int(x) for x in rng.choice(nq, 2, replace=False)) for _ in range(4)]
    for t1, t2 in pairs:
        qs.qs_apply_swap(st.handle, t1, t2)
        want = orc.apply_swap(want, t1, t2)
    got = st.get_amps()
    if prec == 0:
        np.testing.assert_array_equal(got, want.astype(np.complex64))   # moved, not computed: exact
    else:
        np.testing.assert_array_equal(got, want)
    if nq <= 7:
        beta = rand_dm(nq, 3, rng)
        dm = new_dm(qs, nq, prec, beta)
        wantd = beta
        for t1, t2 in pairs:
            qs.qs_apply_swap(dm.handle, t1, t2)
            wantd = orc.densmatr_apply_swap(wantd, t1, t2)
        close(dm.get_amps(), wantd, prec)
    with pytest.raises(qs.QSError) as ei:
        qs.qs_apply_swap(st.handle, 1, 1)
    assert "QS_ERR_DUP_QUBIT" in str(ei.value)
    with pytest.raises(qs.QSError) as ei:
        qs.qs_apply_swap(st.handle, 0, nq)
    assert "QS_ERR_QUBIT_RANGE" in str(ei.value)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n", range(1, 7))
def test_diagonal(qs, prec, n):
    rng = np.random.default_rng(50 + n)
    nq = 11
    targs = [int(x) for x in rng.choice(nq, n, replace=False)]
    d = np.exp(1j * rng.uniform(0, 2 * np.pi, 1 << n)) * rng.uniform(0.5, 1.5, 1 << n)
    psi = wl.random_statevector(nq, rng)
    st = new_sv(qs, nq, prec, psi)
    qs.qs_apply_diagonal(st.handle, targs, d)
    close(st.get_amps(), orc.apply_diagonal(psi, targs, d), prec)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("seed", range(8))
def test_pauli_gadget(qs, prec, seed):
    rng = np.random.default_rng(300 + seed)
    nq = 12
    psi = wl.random_statevector(nq, rng)
    st = new_sv(qs, nq, prec, psi)
    want = psi
    cases = [wl.random_pauli_string(nq, 1, nq, rng) for _ in range(4)]
    cases.append(([0, 5, 11], [3, 3, 3]))            # phase gadget (Z only)
    cases.append(([11], [1]))                        # X on the top qubit
    cases.append(([0, 1], [2, 2]))                   # two Y on the lowest qubits
    cases.append(([], []))                           # global phase exp(-i theta/2)
    for targs, paulis in cases:
        theta = float(rng.uniform(0, 2 * np.pi))
        qs.qs_apply_pauli_gadget(st.handle, targs, paulis, theta)
        want = orc.apply_pauli_gadget(want, targs, paulis, theta)
    close(st.get_amps(), want, prec, scale=4)


@pytest.mark.parametrize("prec", PRECS)
def test_norm_and_statevector_expectation(qs, prec):
    rng = np.random.default_rng(8)
    nq = 11
    psi = wl.random_statevector(nq, rng) * 0.7
    st = new_sv(qs, nq, prec, psi)
    norm = qs.qs_calc_norm_or_trace(st.handle)
    assert abs(norm - orc.calc_norm(psi)) < STOL[prec]
    paulis, coeffs = wl.random_pauli_sum(nq, 13, rng)
    got = qs.qs_expec_pauli_sum(st.handle, paulis, coeffs)
    want = orc.expec_pauli_sum_statevector(psi, paulis, coeffs)
    assert abs(got - want) < STOL[prec] * np.abs(coeffs).sum()
    # terms that share flip masks (grouped by the kernel), diagonal runs, masks whose
    # highest bit is below and above a warp's index span, and repeated strings
    base = wl.random_pauli_sum(nq, 6, rng)[0]
    rows = [base[k % 6].copy() for k in range(30)]
    for k, r in enumerate(rows):
        flips = (r == 1) | (r == 2)
        r[flips] = rng.choice([1, 2], size=int(flips.sum()))   # same X/Y pattern, other Y/X choice
        r[~flips] = rng.choice([0, 3], size=int((~flips).sum()))
    rows += [np.where(np.arange(nq) == q, 1, 0) for q in (0, 3, 4, 5, nq - 1)]
    rows += [np.zeros(nq, dtype=np.int64), np.full(nq, 3)]
    paulis2 = np.array(rows, dtype=np.int32)
    coeffs2 = rng.standard_normal(len(rows))
    got = qs.qs_expec_pauli_sum(st.handle, paulis2, coeffs2)
    want = orc.expec_pauli_sum_statevector(psi, paulis2, coeffs2)
    assert abs(got - want) < STOL[prec] * np.abs(coeffs2).sum()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("nq", [4, 5, 6, 11])
def test_statevector_expectation_many_diagonal_terms(qs, prec, nq):
    """Runs of 40 I/Z strings take the warp Walsh-Hadamard path (N >= 5), with
    masks on every bit including the highest; mixed in are 10 other strings."""
    rng = np.random.default_rng(90 + nq)
    psi = wl.random_statevector(nq, rng)
    st = new_sv(qs, nq, prec, psi)
    zs = np.where(rng.random((40, nq)) < 0.4, 3, 0).astype(np.int32)
    zs[0, :] = 0
    zs[1, :] = 3
    zs[2, :] = 0
    zs[2, nq - 1] = 3
    others = wl.random_pauli_sum(nq, 10, rng)[0]
    paulis = np.concatenate([zs, others])
    coeffs = rng.standard_normal(len(paulis))
    got = qs.qs_expec_pauli_sum(st.handle, paulis, coeffs)
    want = orc.expec_pauli_sum_statevector(psi, paulis, coeffs)
    assert abs(got - want) < STOL[prec] * np.abs(coeffs).sum()
    got_d = qs.qs_expec_pauli_sum(st.handle, zs, coeffs[:40])
    want_d = orc.expec_pauli_sum_statevector(psi, zs, coeffs[:40])
    assert abs(got_d - want_d) < STOL[prec] * np.abs(coeffs[:40]).sum()


@pytest.mark.parametrize("prec", PRECS)
def test_statevector_circuit(qs, prec):
    """500 seeded operations of the 30-qubit workload's mix at 14 qubits."""
    rng = wl.rng_for("sv-circuit-14")
    nq = 14
    psi = wl.random_statevector(nq, rng)
    ops = wl.statevector_circuit(nq, 500, rng)
    st = new_sv(qs, nq, prec, psi)
    for op in ops:
        qs.apply_op(st.handle, op)
    want = orc.run_ops(psi, ops, is_density=False)
    got = st.get_amps()
    if prec:
        err = float(np.max(np.abs(got - want)))
        assert err <= CTOL[prec], err
    else:
        close(got, want, prec, scale=50)
    assert abs(qs.qs_calc_norm_or_trace(st.handle) - 1.0) < (50 * STOL[prec] if prec else 1e-4)


# ---------------------------------------------------------------------------
# density matrices
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", PRECS)
def test_densmatr_init_pure_and_trace(qs, prec):
    rng = np.random.default_rng(21)
    nq = 5
    states, w = wl.random_mixed_state_vectors(nq, 3, rng)
    dm = make_state(qs, nq, True, prec)
    for m, (s, wi) in enumerate(zip(states, w)):
        sv = new_sv(qs, nq, prec, s)
        qs.qs_init_pure_densmatr(dm.handle, sv.handle, wi, accumulate=m > 0)
        qs.qs_synchronize(dm.handle)
        sv.close()
    want = sum(wi * orc.densmatr_from_pure(s) for wi, s in zip(w, states))
    close(dm.get_amps(), want, prec)
    tr = qs.qs_calc_norm_or_trace(dm.handle)
    assert abs(tr - orc.calc_trace(want)) < STOL[prec]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,s", [(1, 0), (1, 2), (2, 0), (2, 3), (3, 1), (3, 3)])
def test_densmatr_unitary(qs, prec, n, s):
    rng = np.random.default_rng(70 + 10 * n + s)
    nq = 6
    beta = rand_dm(nq, 4, rng)
    qsel = [int(x) for x in rng.choice(nq, n + s, replace=False)]
    u = wl.haar_unitary(1 << n, rng)
    dm = new_dm(qs, nq, prec, beta)
    qs.qs_apply_ctrl_multi_target(dm.handle, qsel[n:], qsel[:n], u)
    close(dm.get_amps(), orc.densmatr_apply_ctrl_multi_target(beta, qsel[n:], qsel[:n], u), prec, scale=4)


@pytest.mark.parametrize("prec", PRECS)
def test_densmatr_diag_and_gadget(qs, prec):
    rng = np.random.default_rng(90)
    nq = 6
    beta = rand_dm(nq, 3, rng)
    dm = new_dm(qs, nq, prec, beta)
    want = beta
    d = np.exp(1j * rng.uniform(0, 2 * np.pi, 8))
    qs.qs_apply_diagonal(dm.handle, [4, 0, 2], d)
    want = orc.densmatr_apply_diagonal(want, [4, 0, 2], d)
    for _ in range(6):
        targs, paulis = wl.random_pauli_string(nq, 1, nq, rng)
        theta = float(rng.uniform(0, 2 * np.pi))
        qs.qs_apply_pauli_gadget(dm.handle, targs, paulis, theta)
        want = orc.densmatr_apply_pauli_gadget(want, targs, paulis, theta)
    close(dm.get_amps(), want, prec, scale=4)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("nq,n,m", [(6, 1, 2), (6, 2, 4), (6, 3, 3), (3, 3, 2), (4, 2, 1)])
def test_kraus(qs, prec, nq, n, m):
    rng = np.random.default_rng(110 + nq + n + m)
    beta = rand_dm(nq, 3, rng)
    targs = [int(x) for x in rng.choice(nq, n, replace=False)]
    ks = wl.haar_kraus(n, m, rng)
    dm = new_dm(qs, nq, prec, beta)
    qs.qs_apply_kraus(dm.handle, targs, ks)
    close(dm.get_amps(), orc.densmatr_apply_kraus(beta, targs, ks), prec, scale=4)


CHANNELS = [
    ("dephasing", lambda qs, h, t, p: qs.qs_apply_dephasing(h, t[0], p),
     lambda b, t, p: orc.densmatr_apply_dephasing(b, t[0], p), 1),
    ("dephasing2", lambda qs, h, t, p: qs.qs_apply_two_qubit_dephasing(h, t[0], t[1], p),
     lambda b, t, p: orc.densmatr_apply_two_qubit_dephasing(b, t[0], t[1], p), 2),
    ("depolarising", lambda qs, h, t, p: qs.qs_apply_depolarising(h, t[0], p),
     lambda b, t, p: orc.densmatr_apply_depolarising(b, t[0], p), 1),
    ("depolarising2", lambda qs, h, t, p: qs.qs_apply_two_qubit_depolarising(h, t[0], t[1], p),
     lambda b, t, p: orc.densmatr_apply_two_qubit_depolarising(b, t[0], t[1], p), 2),
    ("damping", lambda qs, h, t, p: qs.qs_apply_damping(h, t[0], p),
     lambda b, t, p: orc.densmatr_apply_damping(b, t[0], p), 1),
    # Pauli channel with (px, py, pz) = (p/2, p/3, p/6) and, for the asymmetric
    # part, (p/5, 0, 3p/5)
    ("pauli", lambda qs, h, t, p: qs.qs_apply_pauli_channel(h, t[0], p / 2, p / 3, p / 6),
     lambda b, t, p: orc.densmatr_apply_pauli_channel(b, t[0], p / 2, p / 3, p / 6), 1),
    ("pauli_xz", lambda qs, h, t, p: qs.qs_apply_pauli_channel(h, t[0], p / 5, 0.0, 3 * p / 5),
     lambda b, t, p: orc.densmatr_apply_pauli_channel(b, t[0], p / 5, 0.0, 3 * p / 5), 1),
]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name,gpu_fn,orc_fn,nt", CHANNELS, ids=[c[0] for c in CHANNELS])
def test_channels(qs, prec, name, gpu_fn, orc_fn, nt):
    rng = np.random.default_rng(sum(ord(c) for c in name))
    nq = 6
    beta = rand_dm(nq, 4, rng)
    dm = new_dm(qs, nq, prec, beta)
    want = beta
    placements = [[int(x) for x in rng.choice(nq, nt, replace=False)] for _ in range(3)]
    placements += [[0, nq - 1][:nt], [nq - 1, 0][:nt]]
    for t in placements:
        p = float(rng.uniform(0, 1))
        gpu_fn(qs, dm.handle, t, p)
        want = orc_fn(want, t, p)
    close(dm.get_amps(), want, prec, scale=4)
    tr = qs.qs_calc_norm_or_trace(dm.handle)
    assert abs(tr - orc.calc_trace(want)) < STOL[prec]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("nq,targs", [(6, [2, 4]), (6, [0]), (6, [5, 0, 3]), (5, [4, 3, 2, 1]), (7, [6, 1])])
def test_partial_trace(qs, prec, nq, targs):
    rng = np.random.default_rng(200 + nq + len(targs))
    beta = rand_dm(nq, 3, rng)
    dm = new_dm(qs, nq, prec, beta)
    red = dm.partial_trace(targs)
    close(red.get_amps(), orc.partial_trace(beta, targs), prec, scale=4)
    # the input is untouched
    close(dm.get_amps(), beta, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_densmatr_expectation(qs, prec):
    rng = np.random.default_rng(31)
    nq = 6
    beta = rand_dm(nq, 4, rng)
    dm = new_dm(qs, nq, prec, beta)
    paulis, coeffs = wl.random_pauli_sum(nq, 20, rng)
    got = qs.qs_expec_pauli_sum(dm.handle, paulis, coeffs)
    want = orc.expec_pauli_sum_densmatr(beta, paulis, coeffs)
    assert abs(got - want) < STOL[prec] * np.abs(coeffs).sum()


@pytest.mark.parametrize("prec", PRECS)
def test_small_density_workload(qs, prec):
    """6-qubit density matrix (12-qubit Choi vector): random mixture of 4
    Gaussian pure states, 300 seeded operations, partial trace over 2 qubits,
    20-term Pauli-sum expectation of the reduced state."""
    rng = wl.rng_for("dm6")
    nq = 6
    states, w = wl.random_mixed_state_vectors(nq, 4, rng)
    ops = wl.small_densmatr_circuit(nq, 300, rng)
    traced = [int(x) for x in rng.choice(nq, 2, replace=False)]
    paulis, coeffs = wl.random_pauli_sum(nq - 2, 20, rng)
    dm = make_state(qs, nq, True, prec)
    for m, (s, wi) in enumerate(zip(states, w)):
        sv = new_sv(qs, nq, prec, s)
        qs.qs_init_pure_densmatr(dm.handle, sv.handle, wi, accumulate=m > 0)
        qs.qs_synchronize(dm.handle)
        sv.close()
    for op in ops:
        qs.apply_op(dm.handle, op)
    red = dm.partial_trace(traced)
    got_e = qs.qs_expec_pauli_sum(red.handle, paulis, coeffs)
    beta = sum(wi * orc.densmatr_from_pure(s) for wi, s in zip(w, states))
    want = orc.run_ops(beta, ops, is_density=True)
    want_red = orc.partial_trace(want, traced)
    want_e = orc.expec_pauli_sum_densmatr(want_red, paulis, coeffs)
    if prec:
        assert float(np.max(np.abs(dm.get_amps() - want))) <= CTOL[prec]
        assert float(np.max(np.abs(red.get_amps() - want_red))) <= CTOL[prec]
        assert abs(got_e - want_e) <= 2 * CTOL[prec] * np.abs(coeffs).sum()
    else:
        close(dm.get_amps(), want, prec, scale=100)
        assert abs(got_e - want_e) <= 1e-4


# ---------------------------------------------------------------------------
# argument validation through a live handle
# ---------------------------------------------------------------------------

def test_validation_errors(qs):
    sv = qs.State(5, density=False)
    qs.qs_init_zero(sv.handle)
    eye = np.eye(2, dtype=np.complex128)
    cases = [
        (lambda: qs.qs_apply_ctrl_multi_target(sv.handle, [], [5], eye), "QS_ERR_QUBIT_RANGE"),
        (lambda: qs.qs_apply_ctrl_multi_target(sv.handle, [1], [1], eye), "QS_ERR_TARGET_IS_CTRL"),
        (lambda: qs.qs_apply_ctrl_multi_target(sv.handle, [2, 2], [1], eye), "QS_ERR_DUP_QUBIT"),
        (lambda: qs.qs_apply_ctrl_multi_target(sv.handle, [], list(range(7)), np.eye(128)), "QS_ERR_TOO_MANY_TARGETS"),
        (lambda: qs.qs_apply_dephasing(sv.handle, 0, 0.1), "QS_ERR_NOT_DENSMATR"),
        (lambda: qs.qs_apply_pauli_gadget(sv.handle, [0], [4], 0.1), "QS_ERR_ARG"),
    ]
    for fn, want in cases:
        with pytest.raises(qs.QSError) as ei:
            fn()
        assert want in str(ei.value)
    dm = qs.State(3, density=True)
    qs.qs_init_zero(dm.handle)
    with pytest.raises(qs.QSError) as ei:
        qs.qs_apply_depolarising(dm.handle, 0, 1.5)
    assert "QS_ERR_ARG" in str(ei.value)
    for probs in ((-0.1, 0.0, 0.0), (0.0, 1.2, 0.0), (0.0, 0.0, float("nan"))):
        with pytest.raises(qs.QSError) as ei:
            qs.qs_apply_pauli_channel(dm.handle, 0, *probs)
        assert "QS_ERR_ARG" in str(ei.value)
    with pytest.raises(qs.QSError) as ei:
        qs.qs_apply_pauli_channel(sv.handle, 0, 0.1, 0.1, 0.1)
    assert "QS_ERR_NOT_DENSMATR" in str(ei.value)
    with pytest.raises(qs.QSError) as ei:
        qs.qs_apply_kraus(dm.handle, [0, 1, 2, 0], [np.eye(16)])
    # nothing changed after the rejected calls
    amps = dm.get_amps()
    assert amps[0] == 1 and np.count_nonzero(amps) == 1
    assert sv.get_amps()[0] == 1


# ---------------------------------------------------------------------------
# tensor-core path (complex64 dense gates, 2..5 targets) against the CUDA cores
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("nq,n,s", [(5, 5, 0), (8, 3, 2), (10, 4, 0), (13, 5, 2), (16, 3, 0), (16, 5, 1),
                                     (3, 2, 0), (4, 2, 1), (11, 2, 2), (17, 4, 1),
                                     (6, 6, 0), (9, 6, 1), (14, 6, 0), (18, 6, 2)])
@pytest.mark.parametrize("place", ["random", "lowest", "highest"])
def test_tensor_core_gate_matches_cuda_cores(qs, nq, n, s, place):
    rng = np.random.default_rng(600 + 10 * nq + n + s + 7 * len(place))
    qsel = [int(x) for x in rng.choice(nq, n + s, replace=False)]
    if place == "lowest":
        qsel = list(range(n + s))
    elif place == "highest":
        qsel = list(range(nq - 1, nq - 1 - n - s, -1))
    targs, ctrls = qsel[:n], qsel[n:]
    psi = wl.random_statevector(nq, rng).astype(np.complex64)
    mat = wl.haar_unitary(1 << n, rng)
    want = orc.apply_ctrl_multi_target(psi.astype(np.complex128), ctrls, targs, mat)
    out = {}
    for tc in (0, 1):
        st = qs.State(nq, prec=0)
        qs.qs_set_tensor_cores(st.handle, tc)
        st.set_amps(psi)
        qs.qs_apply_ctrl_multi_target(st.handle, ctrls, targs, mat)
        qs.qs_synchronize(st.handle)            # also reports a bounded-wait timeout
        out[tc] = st.get_amps().astype(np.complex128)
    scale = float(np.max(np.abs(want)))
    err_cc = float(np.max(np.abs(out[0] - want)))
    err_tc = float(np.max(np.abs(out[1] - want)))
    # 3xTF32 keeps FP32-level accuracy: within 2^-20 of the largest amplitude
    assert err_tc <= scale * 2.0 ** -20, (err_tc, err_cc, scale)


# ---------------------------------------------------------------------------
# complex128 dense gates on the bf16 tensor cores (exact integer slices)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("nq,n,s", [(5, 5, 0), (8, 3, 2), (10, 4, 1), (12, 5, 0), (13, 3, 0), (14, 4, 2),
                                     (3, 2, 0), (4, 2, 1), (9, 2, 3), (13, 2, 0), (16, 5, 1), (17, 3, 1),
                                     (19, 4, 0), (20, 3, 0), (20, 2, 1), (21, 4, 1), (20, 5, 0), (21, 5, 1)])
@pytest.mark.parametrize("kind", ["haar", "wide", "sparse"])
@pytest.mark.parametrize("place", ["random", "lowest", "highest"])
@pytest.mark.parametrize("arith", ["fx", "df"])
def test_complex128_tensor_core_gate(qs, nq, n, s, kind, place, arith):
    """Against the oracle and the CUDA-core double-float kernel.  'wide' uses a
    non-unitary matrix whose entries span 1e-8..1e3 (row and column scaling),
    'sparse' a state that is zero on most groups (all-zero tile rows).  Block
    fixed point runs eight slices (56-bit operands), double-float seven.  Two
    targets run on the three-target kernel with an identity on a free qubit;
    (3, 2, 0) and (4, 2, 1) leave a single free qubit, so the tile has one row.
    Passes of fewer tiles than SMs run the single-CTA kernels; larger 2-4-target
    passes (the 19-21-qubit cases, 256-1024 tiles) the warp-specialised kernel,
    and five targets the single-CTA kernel at every size (here up to 256 tiles)."""
    rng = np.random.default_rng(900 + 31 * nq + 7 * n + s + len(kind) + 3 * len(place))
    qsel = [int(x) for x in rng.choice(nq, n + s, replace=False)]
    if place == "lowest":
        qsel = list(range(n + s))
    elif place == "highest":
        qsel = list(range(nq - 1, nq - 1 - n - s, -1))
    targs, ctrls = qsel[:n], qsel[n:]
    psi = wl.random_statevector(nq, rng)
    mat = wl.haar_unitary(1 << n, rng)
    if kind == "wide":
        mat = mat * 10.0 ** rng.uniform(-8, 3, size=mat.shape)
    if kind == "sparse":
        psi = np.zeros_like(psi)
        psi[rng.choice(psi.size, 5, replace=False)] = rng.standard_normal(5)
    want = orc.apply_ctrl_multi_target(psi, ctrls, targs, mat)
    outs = {}
    for tc in (0, 1):
        st = qs.State(nq, prec=1)
        qs.qs_set_arithmetic(st.handle, qs.QS_ARITH_FX if arith == "fx" else qs.QS_ARITH_DF)
        qs.qs_set_tensor_cores(st.handle, tc)
        st.set_amps(psi)
        qs.qs_apply_ctrl_multi_target(st.handle, ctrls, targs, mat)
        qs.qs_synchronize(st.handle)
        outs[tc] = st.get_amps()
    # error bound of a dot product over K = 2^(n+1) real terms: (K + 1) 2^-54
    # (eight slices) or 2^-47 (seven) of the row and column maxima, here
    # bounded by 2^n max|m| max|psi| times 2^-51 or 2^-44
    ex = -51 if arith == "fx" else -44
    bound = 2.0 ** ex * (np.abs(mat).max() * (1 << n) * np.abs(psi).max()) + 1e-300
    for tc in (0, 1):
        err = float(np.max(np.abs(outs[tc] - want)))
        assert err <= bound, (tc, err, bound)
