"""Pins for the CPU oracle, checked against things other than the oracle
itself: the paper's worked examples (tests/golden/bit_examples.txt), explicit
Kronecker-product operators, scipy's matrix exponential, explicit density
matrices, and invariants the paper states (trace and norm preservation,
Hermiticity, channel fixed points, partial traces of product states).

CPU only.
"""

import os

import numpy as np
import pytest
import scipy.linalg

from oracle import qsim_oracle as orc
from paper_2311_01512_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "bit_examples.txt")

I2 = np.eye(2, dtype=np.complex128)
PX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
PY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
PZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)
PAULI = [I2, PX, PY, PZ]
P1 = np.array([[0, 0], [0, 1]], dtype=np.complex128)


# ---------------------------------------------------------------------------
# Independent constructions: full operators from per-qubit Kronecker factors.
# ---------------------------------------------------------------------------

def kron_list(factors_by_qubit):
    """Operator on N qubits from a list of 2x2 factors, index q = qubit q; the
    Kronecker product runs from qubit N-1 (leftmost) to qubit 0."""
    out = np.array([[1.0 + 0j]])
    for f in reversed(factors_by_qubit):
        out = np.kron(out, f)
    return out


def full_operator(nq, ctrls, targs, mat):
    """1 + P_ctrl (M_ext - 1), with M_ext = sum_rc M[r, c] (x)_q |r_q><c_q| on
    targs[q] (matrix bit q on targs[q]) and identity elsewhere."""
    n = len(targs)
    dim = 1 << n
    m_ext = np.zeros((1 << nq, 1 << nq), dtype=np.complex128)
    for r in range(dim):
        for c in range(dim):
            if mat[r, c] == 0:
                continue
            fac = [I2] * nq
            for q, t in enumerate(targs):
                e = np.zeros((2, 2), dtype=np.complex128)
                e[(r >> q) & 1, (c >> q) & 1] = 1.0
                fac[t] = e
            m_ext += mat[r, c] * kron_list(fac)
    pc = [I2] * nq
    for c in ctrls:
        pc[c] = P1
    proj = kron_list(pc)
    ident = np.eye(1 << nq, dtype=np.complex128)
    return ident + proj @ (m_ext - ident)


def pauli_full(nq, targs, paulis):
    fac = [I2] * nq
    for t, p in zip(targs, paulis):
        fac[t] = PAULI[p]
    return kron_list(fac)


def choi_to_mat(beta):
    dim = int(round(np.sqrt(beta.shape[0])))
    return beta.reshape(dim, dim).T          # beta[k + l dim] = rho[k, l]


def mat_to_choi(rho):
    return np.ascontiguousarray(rho.T).reshape(-1)


def random_density(nq, rank, rng):
    states, w = wl.random_mixed_state_vectors(nq, rank, rng)
    rho = sum(wi * np.outer(s, np.conj(s)) for wi, s in zip(w, states))
    return rho


def ptrace_tensor(rho, nq, traced):
    """Partial trace by contracting tensor axes (rows: axes 0..N-1 for qubits
    N-1..0, columns: axes N..2N-1)."""
    t = rho.reshape([2] * (2 * nq))
    qubits = list(range(nq - 1, -1, -1))          # qubit held by each row axis
    for q in sorted(traced, reverse=True):
        a = qubits.index(q)
        m = len(qubits)
        t = np.trace(t, axis1=a, axis2=a + m)
        qubits.pop(a)
    d = 1 << len(qubits)
    return t.reshape(d, d)


# ---------------------------------------------------------------------------
# Worked examples of the paper (bit-exact).
# ---------------------------------------------------------------------------

def _golden_lines():
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                yield line.split()


def test_golden_worked_examples():
    seen = set()
    for parts in _golden_lines():
        kind = parts[0]
        seen.add(kind)
        if kind == "basis_bits":
            i, nb, bits = int(parts[1]), int(parts[2]), parts[3]
            for pos, ch in enumerate(reversed(bits)):
                assert orc.get_bit(i, pos) == int(ch)
            assert len(bits) == nb
        elif kind == "many_target_index":
            targs = [int(x) for x in parts[1].split(",")]
            nq, k, j, idx = (int(x) for x in parts[2:6])
            base = orc.insert_bits(k, sorted(targs), 0)
            assert orc.set_bits(base, targs, j) == idx
            # the same index through the oracle's vectorised group enumeration:
            # a gate that maps column j to row j' marks exactly that amplitude
            psi = np.zeros(1 << nq, dtype=np.complex128)
            psi[idx] = 1.0
            mat = np.zeros((4, 4), dtype=np.complex128)
            mat[0, j] = 1.0                        # |j> -> |0> on the targets
            out = orc.apply_ctrl_multi_target(psi, [], targs, mat)
            assert np.flatnonzero(out).tolist() == [orc.insert_bits(k, sorted(targs), 0)]
        elif kind == "complement":
            nb, i, ci = (int(x) for x in parts[1:4])
            assert orc.flip_bits(i, range(nb)) == ci
        elif kind == "ptrace_layout":
            nq = int(parts[1])
            targs = [int(x) for x in parts[2].split(",")]
            vpos = [int(x) for x in parts[3].split(",")]
            ipos = [int(x) for x in parts[4].split(",")]
            traced = sorted(targs + [t + nq for t in targs])
            assert traced == vpos
            kept = sorted(set(range(2 * nq)) - set(traced))
            assert kept == ipos
            # The oracle's partial trace reads exactly the amplitudes g(i, v):
            # mark one Choi amplitude with v bits equal on t and t+N and check
            # which output it lands in.
            rho = np.zeros(1 << (2 * nq), dtype=np.complex128)
            i_val, v_val = 0b101101, 0b10
            g = 0
            for q, p in enumerate(ipos):
                g |= ((i_val >> q) & 1) << p
            vv = (v_val << len(targs)) | v_val
            for q, p in enumerate(targs + [t + nq for t in targs]):
                g |= ((vv >> q) & 1) << p
            rho[g] = 1.0
            out = orc.partial_trace(rho, targs)
            assert np.flatnonzero(out).tolist() == [i_val]
    assert seen == {"basis_bits", "many_target_index", "complement", "ptrace_layout"}


def test_insert_bit_and_masks():
    assert orc.insert_bit(0b1011, 2, 1) == 0b10111
    assert orc.insert_bit(0b1011, 0, 0) == 0b10110
    assert orc.get_bit_mask([0, 3, 5]) == 0b101001
    assert orc.all_bits_are_one(0b101001, [0, 3, 5]) == 1
    assert orc.all_bits_are_one(0b100001, [0, 3, 5]) == 0
    for x in range(256):
        assert orc.mask_parity(x) == bin(x).count("1") % 2
    xs = np.arange(1 << 12, dtype=np.int64) * 7919
    assert np.array_equal(orc._v_parity(xs), np.array([bin(int(x)).count("1") & 1 for x in xs]))


# ---------------------------------------------------------------------------
# Statevector gates against full Kronecker-built operators (N <= 8).
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("nq,ntarg,nctrl", [(1, 1, 0), (3, 1, 0), (5, 1, 2), (6, 2, 0), (6, 2, 3),
                                            (7, 3, 2), (8, 4, 1), (8, 1, 7 - 0), (6, 6, 0)])
def test_gate_matches_kronecker(nq, ntarg, nctrl):
    rng = np.random.default_rng(nq * 100 + ntarg * 10 + nctrl)
    nctrl = min(nctrl, nq - ntarg)
    for trial in range(3):
        qs = [int(x) for x in rng.choice(nq, ntarg + nctrl, replace=False)]
        targs, ctrls = qs[:ntarg], qs[ntarg:]
        # a general (non-unitary) matrix: the method does not need unitarity
        mat = rng.standard_normal((1 << ntarg, 1 << ntarg)) + 1j * rng.standard_normal((1 << ntarg, 1 << ntarg))
        psi = rng.standard_normal(1 << nq) + 1j * rng.standard_normal(1 << nq)
        want = full_operator(nq, ctrls, targs, mat) @ psi
        got = orc.apply_ctrl_multi_target(psi, ctrls, targs, mat)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def test_one_target_gate_equals_kron_identity_u_identity():
    rng = np.random.default_rng(7)
    nq = 5
    u = wl.haar_unitary(2, rng)
    psi = wl.random_statevector(nq, rng)
    for t in range(nq):
        full = np.kron(np.kron(np.eye(1 << (nq - t - 1)), u), np.eye(1 << t))
        np.testing.assert_allclose(orc.apply_ctrl_multi_target(psi, [], [t], u), full @ psi, atol=1e-13)


def test_diagonal_matches_kronecker():
    rng = np.random.default_rng(11)
    nq = 7
    for n in (1, 2, 3):
        targs = [int(x) for x in rng.choice(nq, n, replace=False)]
        d = np.exp(1j * rng.uniform(0, 2 * np.pi, 1 << n))
        psi = wl.random_statevector(nq, rng)
        want = full_operator(nq, [], targs, np.diag(d)) @ psi
        np.testing.assert_allclose(orc.apply_diagonal(psi, targs, d), want, atol=1e-13)


@pytest.mark.parametrize("seed", range(6))
def test_pauli_gadget_closed_form_and_expm(seed):
    rng = np.random.default_rng(seed)
    nq = 6
    targs, paulis = wl.random_pauli_string(nq, 1, nq, rng)
    theta = float(rng.uniform(0, 2 * np.pi))
    pf = pauli_full(nq, targs, paulis)
    closed = np.cos(theta / 2) * np.eye(1 << nq) - 1j * np.sin(theta / 2) * pf
    np.testing.assert_allclose(closed, scipy.linalg.expm(-0.5j * theta * pf), atol=1e-12)
    psi = wl.random_statevector(nq, rng)
    np.testing.assert_allclose(orc.apply_pauli_gadget(psi, targs, paulis, theta), closed @ psi, atol=1e-13)
    np.testing.assert_allclose(orc.apply_pauli_tensor(psi, targs, paulis), pf @ psi, atol=1e-13)


def test_phase_gadget_is_parity_phase():
    # Z-only gadget: alpha_i -> exp(i phi s_i) alpha_i with phi = -theta/2,
    # s_i = +1 for even parity of the targeted bits (Sec. "Phase gadget").
    nq, theta = 5, 0.7
    targs = [0, 3, 4]
    psi = np.ones(1 << nq, dtype=np.complex128)
    out = orc.apply_pauli_gadget(psi, targs, [3, 3, 3], theta)
    for i in range(1 << nq):
        par = sum((i >> t) & 1 for t in targs) % 2
        assert abs(out[i] - np.exp(1j * (-theta / 2) * (1 if par == 0 else -1))) < 1e-15


def test_norm_and_statevector_expectation():
    rng = np.random.default_rng(3)
    nq = 6
    psi = wl.random_statevector(nq, rng)
    assert abs(orc.calc_norm(psi) - 1.0) < 1e-13
    for op in wl.unitary_circuit(nq, 40, rng):
        if op["op"] == "unitary":
            psi = orc.apply_ctrl_multi_target(psi, op["ctrls"], op["targs"], op["mat"])
        else:
            psi = orc.apply_pauli_gadget(psi, op["targs"], op["paulis"], op["theta"])
    assert abs(orc.calc_norm(psi) - 1.0) < 1e-12
    paulis, coeffs = wl.random_pauli_sum(nq, 7, rng)
    h = sum(c * pauli_full(nq, list(range(nq)), [int(x) for x in row]) for row, c in zip(paulis, coeffs))
    want = np.vdot(psi, h @ psi)
    got = orc.expec_pauli_sum_statevector(psi, paulis, coeffs)
    assert abs(got - want) < 1e-12
    assert abs(got.imag) < 1e-12


# ---------------------------------------------------------------------------
# Density matrices against explicit matrices (N <= 4).
# ---------------------------------------------------------------------------

def test_choi_layout_matches_paper():
    rng = np.random.default_rng(0)
    psi = wl.random_statevector(3, rng)
    beta = orc.densmatr_from_pure(psi)
    # beta_{j + k 2^N} = psi_j psi_k^*  (pure-state initialisation)
    for j in range(8):
        for k in range(8):
            assert abs(beta[j + 8 * k] - psi[j] * np.conj(psi[k])) < 1e-15
    rho = np.outer(psi, np.conj(psi))
    np.testing.assert_allclose(choi_to_mat(beta), rho, atol=1e-15)
    np.testing.assert_allclose(orc.densmatr_from_matrix(rho), beta, atol=1e-15)
    np.testing.assert_allclose(orc.densmatr_to_matrix(beta), rho, atol=1e-15)
    assert abs(orc.calc_trace(beta) - 1.0) < 1e-14


@pytest.mark.parametrize("seed", range(4))
def test_densmatr_unitary_and_gadget(seed):
    rng = np.random.default_rng(100 + seed)
    nq = 4
    rho = random_density(nq, 3, rng)
    beta = mat_to_choi(rho)
    targs = [int(x) for x in rng.choice(nq, 3, replace=False)]
    u = wl.haar_unitary(4, rng)
    uf = full_operator(nq, [targs[2]], targs[:2], u)
    got = choi_to_mat(orc.densmatr_apply_ctrl_multi_target(beta, [targs[2]], targs[:2], u))
    np.testing.assert_allclose(got, uf @ rho @ uf.conj().T, atol=1e-13)
    gt, gp = wl.random_pauli_string(nq, 1, nq, rng)
    theta = float(rng.uniform(0, 2 * np.pi))
    gf = scipy.linalg.expm(-0.5j * theta * pauli_full(nq, gt, gp))
    got = choi_to_mat(orc.densmatr_apply_pauli_gadget(beta, gt, gp, theta))
    np.testing.assert_allclose(got, gf @ rho @ gf.conj().T, atol=1e-12)
    d = np.exp(1j * rng.uniform(0, 2 * np.pi, 4))
    df = full_operator(nq, [], targs[:2], np.diag(d))
    got = choi_to_mat(orc.densmatr_apply_diagonal(beta, targs[:2], d))
    np.testing.assert_allclose(got, df @ rho @ df.conj().T, atol=1e-13)


SWAP4 = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)
XMAT = np.array([[0, 1], [1, 0]], dtype=np.complex128)


def test_swap_pins():
    """SWAP (Sec. "Swap gate") against its 4x4 matrix as a two-target gate, three
    CNOTs, an explicit basis-state example, the Kronecker operator, and S rho S
    on a density matrix."""
    rng = np.random.default_rng(61)
    nq = 5
    # worked example: |0b00001> with t1 = 0, t2 = 4 becomes |0b10000>
    e = np.zeros(1 << nq, dtype=np.complex128)
    e[0b00001] = 1.0
    out = orc.apply_swap(e, 0, 4)
    assert out[0b10000] == 1.0 and np.count_nonzero(out) == 1
    psi = wl.random_statevector(nq, rng)
    for t1, t2 in ((0, 4), (3, 1), (2, 3)):
        got = orc.apply_swap(psi, t1, t2)
        np.testing.assert_allclose(got, orc.apply_ctrl_multi_target(psi, [], [t1, t2], SWAP4), atol=0)
        cn = orc.apply_ctrl_multi_target(psi, [t1], [t2], XMAT)
        cn = orc.apply_ctrl_multi_target(cn, [t2], [t1], XMAT)
        cn = orc.apply_ctrl_multi_target(cn, [t1], [t2], XMAT)
        np.testing.assert_allclose(got, cn, atol=0)
        np.testing.assert_allclose(got, full_operator(nq, [], [t1, t2], SWAP4) @ psi, atol=1e-15)
        np.testing.assert_allclose(orc.apply_swap(got, t2, t1), psi, atol=0)
    got = orc.apply_swap(psi, 1, 4)
    idx = np.arange(1 << nq)
    np.testing.assert_array_equal(orc.sample_swap(lambda ix: psi[np.asarray(ix)], 1, 4, idx), got)
    rho = random_density(4, 3, rng)
    sw = full_operator(4, [], [0, 2], SWAP4)
    np.testing.assert_allclose(choi_to_mat(orc.densmatr_apply_swap(mat_to_choi(rho), 0, 2)), sw @ rho @ sw,
                               atol=1e-15)


def test_superoperator_of_one_unitary_is_two_pass_unitary():
    rng = np.random.default_rng(5)
    nq = 3
    beta = mat_to_choi(random_density(nq, 2, rng))
    u = wl.haar_unitary(4, rng)
    a = orc.densmatr_apply_kraus(beta, [2, 0], [u])
    b = orc.densmatr_apply_ctrl_multi_target(beta, [], [2, 0], u)
    np.testing.assert_allclose(a, b, atol=1e-13)
    # S = conj(K) (x) K as a standard Kronecker product
    k = wl.haar_kraus(1, 2, rng)
    s = orc.superoperator(k)
    np.testing.assert_allclose(s, np.kron(k[0].conj(), k[0]) + np.kron(k[1].conj(), k[1]), atol=0)


@pytest.mark.parametrize("nk", [1, 2])
def test_kraus_matches_explicit(nk):
    rng = np.random.default_rng(20 + nk)
    nq = 4
    rho = random_density(nq, 3, rng)
    targs = [int(x) for x in rng.choice(nq, nk, replace=False)]
    ks = wl.haar_kraus(nk, 4, rng)
    want = sum(full_operator(nq, [], targs, k) @ rho @ full_operator(nq, [], targs, k).conj().T for k in ks)
    got = choi_to_mat(orc.densmatr_apply_kraus(mat_to_choi(rho), targs, ks))
    np.testing.assert_allclose(got, want, atol=1e-13)
    assert abs(np.trace(got) - 1.0) < 1e-13            # trace preserved (sum K^dag K = 1)


def _paulis_on(nq, t, p):
    return pauli_full(nq, [t], [p])


@pytest.mark.parametrize("seed", range(3))
def test_channels_match_explicit(seed):
    rng = np.random.default_rng(40 + seed)
    nq = 4
    rho = random_density(nq, 4, rng)
    beta = mat_to_choi(rho)
    t, t2 = [int(x) for x in rng.choice(nq, 2, replace=False)]
    p = float(rng.uniform(0, 0.3))
    z1, z2 = _paulis_on(nq, t, 3), _paulis_on(nq, t2, 3)
    want = (1 - p) * rho + p * z1 @ rho @ z1
    np.testing.assert_allclose(choi_to_mat(orc.densmatr_apply_dephasing(beta, t, p)), want, atol=1e-14)
    want = (1 - p) * rho + p / 3 * (z1 @ rho @ z1 + z2 @ rho @ z2 + z1 @ z2 @ rho @ z2 @ z1)
    np.testing.assert_allclose(choi_to_mat(orc.densmatr_apply_two_qubit_dephasing(beta, t, t2, p)), want, atol=1e-14)
    want = (1 - p) * rho + p / 3 * sum(_paulis_on(nq, t, k) @ rho @ _paulis_on(nq, t, k) for k in (1, 2, 3))
    np.testing.assert_allclose(choi_to_mat(orc.densmatr_apply_depolarising(beta, t, p)), want, atol=1e-14)
    acc = np.zeros_like(rho)
    for a in range(4):
        for b in range(4):
            s = _paulis_on(nq, t, a) @ _paulis_on(nq, t2, b)
            acc += s @ rho @ s.conj().T
    want = (1 - 16 * p / 15) * rho + p / 15 * acc
    got = choi_to_mat(orc.densmatr_apply_two_qubit_depolarising(beta, t, t2, p))
    np.testing.assert_allclose(got, want, atol=1e-14)
    k1 = full_operator(nq, [], [t], np.array([[1, 0], [0, np.sqrt(1 - p)]]))
    k2 = full_operator(nq, [], [t], np.array([[0, np.sqrt(p)], [0, 0]]))
    want = k1 @ rho @ k1.conj().T + k2 @ rho @ k2.conj().T
    np.testing.assert_allclose(choi_to_mat(orc.densmatr_apply_damping(beta, t, p)), want, atol=1e-14)


@pytest.mark.parametrize("seed", range(3))
def test_pauli_channel_matches_explicit_and_special_cases(seed):
    """General one-qubit Pauli channel: explicit Pauli conjugations of the
    density matrix, its Kraus form, and its depolarising (p/3 each) and
    dephasing (0, 0, p) special cases, which come from other equations."""
    rng = np.random.default_rng(300 + seed)
    nq = 4
    rho = random_density(nq, 4, rng)
    beta = mat_to_choi(rho)
    t = int(rng.integers(nq))
    px, py, pz = (float(x) for x in rng.uniform(0, 0.3, 3))
    want = (1 - px - py - pz) * rho
    for p, k in ((px, 1), (py, 2), (pz, 3)):
        s = _paulis_on(nq, t, k)
        want = want + p * s @ rho @ s.conj().T
    got = orc.densmatr_apply_pauli_channel(beta, t, px, py, pz)
    np.testing.assert_allclose(choi_to_mat(got), want, atol=1e-14)
    kraus = [np.sqrt(1 - px - py - pz) * I2, np.sqrt(px) * np.array([[0, 1], [1, 0]]),
             np.sqrt(py) * np.array([[0, -1j], [1j, 0]]), np.sqrt(pz) * np.array([[1, 0], [0, -1]])]
    np.testing.assert_allclose(got, orc.densmatr_apply_kraus(beta, [t], kraus), atol=1e-14)
    p = float(rng.uniform(0, 0.5))
    np.testing.assert_allclose(orc.densmatr_apply_pauli_channel(beta, t, p / 3, p / 3, p / 3),
                               orc.densmatr_apply_depolarising(beta, t, p), atol=1e-15)
    np.testing.assert_allclose(orc.densmatr_apply_pauli_channel(beta, t, 0, 0, p),
                               orc.densmatr_apply_dephasing(beta, t, p), atol=1e-15)
    # bit flip with px = 1/2 and phase flip with pz = 1/2 remove the X / Z coherences:
    # together they replace qubit t by I/2 (an independent fixed point)
    twice = orc.densmatr_apply_pauli_channel(orc.densmatr_apply_pauli_channel(beta, t, 0.5, 0, 0), t, 0, 0, 0.5)
    np.testing.assert_allclose(choi_to_mat(twice), choi_to_mat(orc.densmatr_apply_depolarising(beta, t, 0.75)),
                               atol=1e-14)


def test_channel_fixed_points_and_special_cases():
    rng = np.random.default_rng(77)
    nq = 3
    rho = random_density(nq, 3, rng)
    beta = mat_to_choi(rho)
    top = nq - 1
    # one-qubit depolarising at p = 3/4 replaces qubit t by I/2
    got = choi_to_mat(orc.densmatr_apply_depolarising(beta, top, 0.75))
    np.testing.assert_allclose(got, np.kron(I2 / 2, ptrace_tensor(rho, nq, [top])), atol=1e-14)
    got = choi_to_mat(orc.densmatr_apply_depolarising(beta, 0, 0.75))
    np.testing.assert_allclose(got, np.kron(ptrace_tensor(rho, nq, [0]), I2 / 2), atol=1e-14)
    # two-qubit depolarising at p = 15/16 replaces both qubits by I/4
    got = choi_to_mat(orc.densmatr_apply_two_qubit_depolarising(beta, 1, 2, 15 / 16))
    np.testing.assert_allclose(got, np.kron(np.eye(4) / 4, ptrace_tensor(rho, nq, [1, 2])), atol=1e-14)
    # damping at p = 1 sends the qubit to |0><0|
    got = choi_to_mat(orc.densmatr_apply_damping(beta, top, 1.0))
    zero = np.array([[1, 0], [0, 0]], dtype=np.complex128)
    np.testing.assert_allclose(got, np.kron(zero, ptrace_tensor(rho, nq, [top])), atol=1e-14)
    # the maximally mixed state is a fixed point of dephasing and depolarising
    mm = mat_to_choi(np.eye(1 << nq) / (1 << nq))
    for f in (lambda b: orc.densmatr_apply_dephasing(b, 1, 0.3),
              lambda b: orc.densmatr_apply_two_qubit_dephasing(b, 0, 2, 0.4),
              lambda b: orc.densmatr_apply_depolarising(b, 2, 0.2),
              lambda b: orc.densmatr_apply_two_qubit_depolarising(b, 0, 1, 0.5)):
        np.testing.assert_allclose(f(mm), mm, atol=1e-16)


def test_partial_trace_of_products_and_random():
    rng = np.random.default_rng(9)
    singles = [random_density(1, 2, rng) for _ in range(4)]   # qubit q -> singles[q]
    rho = kron_list(singles)
    beta = mat_to_choi(rho)
    # trace out qubits {0, 2}: the rest keep their order, qubit 3 above qubit 1
    got = choi_to_mat(orc.partial_trace(beta, [2, 0]))
    np.testing.assert_allclose(got, np.kron(singles[3], singles[1]), atol=1e-15)
    got = choi_to_mat(orc.partial_trace(beta, [3]))
    np.testing.assert_allclose(got, kron_list(singles[:3]), atol=1e-15)
    for nq, traced in ((4, [1, 3]), (5, [0, 4, 2]), (3, [1])):
        r = random_density(nq, 3, rng)
        got = choi_to_mat(orc.partial_trace(mat_to_choi(r), traced))
        np.testing.assert_allclose(got, ptrace_tensor(r, nq, traced), atol=1e-15)
        assert abs(np.trace(got) - np.trace(r)) < 1e-14


def test_densmatr_expectation():
    rng = np.random.default_rng(12)
    nq = 4
    rho = random_density(nq, 3, rng)
    beta = mat_to_choi(rho)
    paulis, coeffs = wl.random_pauli_sum(nq, 9, rng)
    h = sum(c * pauli_full(nq, list(range(nq)), [int(x) for x in row]) for row, c in zip(paulis, coeffs))
    want = np.trace(h @ rho)
    got = orc.expec_pauli_sum_densmatr(beta, paulis, coeffs)
    assert abs(got - want) < 1e-13
    assert abs(got.imag) < 1e-13
    # special cases: Z_q on |0><0| gives 1; the identity string gives Tr rho
    zero = mat_to_choi(np.diag([1.0] + [0.0] * ((1 << nq) - 1)).astype(np.complex128))
    zq = np.zeros((1, nq), dtype=np.int32)
    zq[0, 2] = 3
    assert abs(orc.expec_pauli_sum_densmatr(zero, zq, [1.0]) - 1.0) < 1e-15
    assert abs(orc.expec_pauli_sum_densmatr(beta, np.zeros((1, nq), dtype=np.int32), [1.0]) - np.trace(rho)) < 1e-14


def test_random_noisy_circuit_keeps_trace_and_hermiticity():
    rng = np.random.default_rng(2)
    nq = 4
    states, w = wl.random_mixed_state_vectors(nq, 4, rng)
    beta = sum(wi * orc.densmatr_from_pure(s) for wi, s in zip(w, states))
    ops = wl.small_densmatr_circuit(nq, 60, rng)
    out = orc.run_ops(beta, ops, is_density=True)
    rho = choi_to_mat(out)
    assert abs(np.trace(rho) - 1.0) < 1e-12
    np.testing.assert_allclose(rho, rho.conj().T, atol=1e-13)
    assert np.min(np.linalg.eigvalsh(rho)) > -1e-12


def test_single_amplitude_oracle_matches_whole_state():
    rng = np.random.default_rng(321)
    nq = 9
    psi = wl.random_statevector(nq, rng)
    get = lambda idx: psi[np.asarray(idx)]
    out_idx = rng.choice(1 << nq, 40, replace=False)
    for n, s in ((1, 0), (2, 2), (4, 1), (5, 0)):
        qsel = [int(x) for x in rng.choice(nq, n + s, replace=False)]
        mat = rng.standard_normal((1 << n, 1 << n)) + 1j * rng.standard_normal((1 << n, 1 << n))
        want = orc.apply_ctrl_multi_target(psi, qsel[n:], qsel[:n], mat)[out_idx]
        got = orc.sample_ctrl_multi_target(get, qsel[n:], qsel[:n], mat, out_idx)
        np.testing.assert_allclose(got, want, atol=1e-13)
    d = np.exp(1j * rng.uniform(0, 6, 8))
    np.testing.assert_allclose(orc.sample_diagonal(get, [3, 0, 7], d, out_idx),
                               orc.apply_diagonal(psi, [3, 0, 7], d)[out_idx], atol=1e-15)
    targs, paulis = wl.random_pauli_string(nq, 1, nq, rng)
    np.testing.assert_allclose(orc.sample_pauli_gadget(get, targs, paulis, 0.9, out_idx),
                               orc.apply_pauli_gadget(psi, targs, paulis, 0.9)[out_idx], atol=1e-15)


@pytest.mark.parametrize("nq", [2, 3, 4])
def test_sampled_channels_match_full_channels(nq):
    """The single-output channel forms (used where a Choi vector is too large
    for the whole-vector oracle) give the whole-vector channels' result at
    every index, for every qubit placement."""
    rng = np.random.default_rng(40 + nq)
    beta = rng.standard_normal(1 << (2 * nq)) + 1j * rng.standard_normal(1 << (2 * nq))
    get = lambda ix: beta[np.asarray(ix)]
    idx = np.arange(beta.size)
    p = float(rng.uniform(0, 1))
    probs = rng.uniform(0, 0.3, 3)
    for t in range(nq):
        pairs = [
            (orc.densmatr_apply_dephasing(beta, t, p), orc.sample_densmatr_dephasing(get, nq, t, p, idx)),
            (orc.densmatr_apply_depolarising(beta, t, p), orc.sample_densmatr_depolarising(get, nq, t, p, idx)),
            (orc.densmatr_apply_damping(beta, t, p), orc.sample_densmatr_damping(get, nq, t, p, idx)),
            (orc.densmatr_apply_pauli_channel(beta, t, *probs),
             orc.sample_densmatr_pauli_channel(get, nq, t, *probs, idx)),
        ]
        for t2 in range(nq):
            if t2 == t:
                continue
            pairs.append((orc.densmatr_apply_two_qubit_dephasing(beta, t, t2, p),
                          orc.sample_densmatr_two_qubit_dephasing(get, nq, t, t2, p, idx)))
            pairs.append((orc.densmatr_apply_two_qubit_depolarising(beta, t, t2, p),
                          orc.sample_densmatr_two_qubit_depolarising(get, nq, t, t2, p, idx)))
        for full, sampled in pairs:
            np.testing.assert_allclose(sampled, full, rtol=0, atol=1e-14)
