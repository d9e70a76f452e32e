"""CPU oracle for the local full-state hot path of "Distributed Simulation of
Statevectors and Density Matrices" (arXiv 2311.01512).

TEST INFRASTRUCTURE ONLY.  This module is a plain, slow, complex128 restatement
of the paper's local operations, written to check the CUDA path.  Only the test
suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl
reference`` legs of ``bench.py`` may import it.  The library never calls it,
and it shares no code with the CUDA path: it imports nothing from the package.

Conventions (paper, Sec. "Notation"): qubit 0 is the least significant bit of
a basis index; a statevector of N qubits is a complex array of 2^N amplitudes;
bit q of a gate-matrix index belongs to target ``targs[q]`` (Sec. "Many-target
gate").  A density matrix rho = sum_kl alpha_kl |k><l| of N qubits is held as
its Choi vector of 2N qubits, beta_i = alpha_{i mod 2^N, floor(i / 2^N)}
(Sec. "State representation").

Every function below cites the passage it follows.  Each takes the whole
state as a numpy array and returns a new array (the input is not modified).

Pinned by ``tests/test_oracle_pins.py`` against the paper's worked examples,
explicit Kronecker-product matrices, scipy's ``expm``, explicit density
matrices, and the invariants the paper states.
"""

import numpy as np

# --------------------------------------------------------------------------
# Bit twiddling (Algorithm "bit twiddles", Sec. "Notation").  Plain Python
# integers, so that the worked examples of the paper can be checked exactly.
# --------------------------------------------------------------------------


def get_bit(n, t):
    """Bit t of n (Algorithm "bit twiddles": getBit)."""
    return (n >> t) & 1


def flip_bit(n, t):
    """n with bit t flipped (Algorithm "bit twiddles": flipBit)."""
    return n ^ (1 << t)


def flip_bits(n, ts):
    """n with every bit in ts flipped (Algorithm "bit twiddles": flipBits)."""
    for q in ts:
        n = flip_bit(n, q)
    return n


def insert_bit(n, t, b):
    """Insert bit value b at position t, shifting higher bits up by one
    (Algorithm "bit twiddles": insertBit)."""
    left = (n >> t) << (t + 1)
    mid = b << t
    right = n & ((1 << t) - 1)
    return left | mid | right


def insert_bits(n, ts, b):
    """Insert bit value b at each of the sorted positions ts, lowest first
    (Algorithm "bit twiddles": insertBits; ts must be sorted)."""
    for q in ts:
        n = insert_bit(n, q, b)
    return n


def set_bits(n, ts, v):
    """Set bit ts[q] of n when bit q of v is 1 (Algorithm "bit twiddles":
    setBits).  As in the paper, the bits at ts are expected to be zero on
    entry (they are, after insertBits with b = 0)."""
    for q in range(len(ts)):
        b = get_bit(v, q) << ts[q]
        n = (n & ~b) | b
    return n


def all_bits_are_one(n, ts):
    """1 if every bit of n at the positions ts is 1 (Algorithm "bit twiddles":
    allBitsAreOne)."""
    v = 1
    for q in ts:
        v &= get_bit(n, q)
    return v


def get_bit_mask(ts):
    """Mask with the bits ts set (Algorithm "bit twiddles": getBitMask)."""
    return flip_bits(0, ts)


def mask_parity(x):
    """Parity of the number of set bits of x.  The paper names getMaskParity
    (Sec. "Phase gadget") without defining it; it is the popcount mod 2."""
    return bin(x).count("1") & 1


# Vectorised forms of the same primitives over numpy uint64 index arrays.  Each
# is the scalar rule above applied elementwise.

def _v_insert_bits(k, ts_sorted, b):
    """Elementwise insertBits over an int64 array of group numbers k."""
    n = k.astype(np.int64)
    for q in ts_sorted:
        left = (n >> q) << (q + 1)
        right = n & ((1 << q) - 1)
        n = left | (b << q) | right
    return n


def _v_set_bits_offsets(ts, nbits_v):
    """offsets[v] = setBits(0, ts, v) for every v < 2^len(ts)."""
    return np.array([set_bits(0, ts, v) for v in range(1 << nbits_v)], dtype=np.int64)


def _v_parity(x):
    """Elementwise parity of the set bits of a non-negative int64 array."""
    x = x.astype(np.uint64)
    for s in (32, 16, 8, 4, 2, 1):
        x = x ^ (x >> np.uint64(s))
    return (x & np.uint64(1)).astype(np.int64)


def _num_qubits(state):
    n = int(state.shape[0]).bit_length() - 1
    if (1 << n) != state.shape[0]:
        raise ValueError("state length is not a power of two")
    return n


def _check_qubits(nq, qubits):
    qs = list(qubits)
    if len(set(qs)) != len(qs):
        raise ValueError("duplicate qubit")
    for q in qs:
        if not 0 <= q < nq:
            raise ValueError("qubit out of range")


# --------------------------------------------------------------------------
# Statevector operations (Sec. "Local statevector algorithms")
# --------------------------------------------------------------------------


def apply_ctrl_multi_target(psi, ctrls, targs, mat):
    """Many-control many-target dense gate on a statevector (or on a Choi
    vector treated as one).

    Sec. "Many-target gate", Eq. (local many-target amplitude update):
    alpha_{kj} -> sum_l m_{jl} alpha_{kl}, where j runs over the 2^n values of
    the target bits (bit q of j on qubit targs[q]) and k over the assignments
    of the other qubits.  Sec. "Many-control one-target gate", Eq. (control
    condition): only the amplitudes whose control bits are all 1 change.
    The matrix need not be unitary.
    """
    psi = np.array(psi, dtype=np.complex128, copy=True)
    nq = _num_qubits(psi)
    ctrls, targs = list(ctrls), list(targs)
    _check_qubits(nq, ctrls + targs)
    n = len(targs)
    mat = np.asarray(mat, dtype=np.complex128)
    if mat.shape != (1 << n, 1 << n):
        raise ValueError("matrix shape does not match the targets")
    fixed = sorted(ctrls + targs)
    num_groups = 1 << (nq - len(fixed))
    k = np.arange(num_groups, dtype=np.int64)
    # group base index: zero bits at every target and control position, then
    # the control bits set to one
    base = _v_insert_bits(k, fixed, 0) | get_bit_mask(ctrls)
    offsets = _v_set_bits_offsets(targs, n)
    idx = base[:, None] | offsets[None, :]          # idx[k, j] holds alpha_{kj}
    old = psi[idx]
    psi[idx] = old @ mat.T                          # new[k, j] = sum_l m[j, l] old[k, l]
    return psi


def apply_swap(psi, t1, t2):
    """SWAP of qubits t1, t2 (Sec. "Swap gate"): alpha_i -> alpha_{i with
    bits t1 and t2 flipped} where bits t1 and t2 of i differ, else alpha_i."""
    psi = np.asarray(psi, dtype=np.complex128)
    i = np.arange(psi.shape[0], dtype=np.int64)
    differ = ((i >> t1) & 1) != ((i >> t2) & 1)
    return np.where(differ, psi[i ^ ((1 << t1) | (1 << t2))], psi)


def densmatr_apply_swap(rho, t1, t2):
    """SWAP on a Choi vector (Sec. "Unitary gates"): SWAP on (t1, t2) and,
    SWAP being real, SWAP again on (t1 + N, t2 + N)."""
    nq = _dm_qubits(rho)
    return apply_swap(apply_swap(rho, t1, t2), t1 + nq, t2 + nq)


def apply_diagonal(psi, targs, diag):
    """Diagonal n-target operator: alpha_i -> d_j alpha_i, with j the value of
    the target bits of i (bit q of j on qubit targs[q]).  This is the
    many-target update of Sec. "Many-target gate" with a diagonal matrix; the
    phase gadget of Sec. "Phase gadget" is the case d_j = exp(i theta s_j)."""
    psi = np.array(psi, dtype=np.complex128, copy=True)
    nq = _num_qubits(psi)
    targs = list(targs)
    _check_qubits(nq, targs)
    diag = np.asarray(diag, dtype=np.complex128)
    i = np.arange(1 << nq, dtype=np.int64)
    j = np.zeros_like(i)
    for q, t in enumerate(targs):
        j |= ((i >> t) & 1) << q
    return psi * diag[j]


def _pauli_masks(targs, paulis):
    """x-flip mask (qubits with X or Y), y/z-sign mask (qubits with Y or Z) and
    the number of Y factors.  Pauli codes: 0 = I, 1 = X, 2 = Y, 3 = Z."""
    xy = yz = 0
    num_y = 0
    for t, p in zip(targs, paulis):
        if p not in (0, 1, 2, 3):
            raise ValueError("Pauli code must be 0..3")
        if p in (1, 2):
            xy |= 1 << t
        if p in (2, 3):
            yz |= 1 << t
        if p == 2:
            num_y += 1
    return xy, yz, num_y


def apply_pauli_tensor(psi, targs, paulis):
    """Pauli tensor (Sec. "Pauli tensor", Eq. (Pauli tensor amplitude
    update)): alpha_i -> beta_{i'} alpha_{i'}, with i' = i with the X/Y
    target bits flipped, beta_i = (-1)^{f(i)} eta, eta = i^{#Y}, and f(i) the
    number of Y/Z targets whose bit in i is 1."""
    psi = np.asarray(psi, dtype=np.complex128)
    nq = _num_qubits(psi)
    _check_qubits(nq, targs)
    xy, yz, num_y = _pauli_masks(targs, paulis)
    eta = 1j ** num_y
    i = np.arange(1 << nq, dtype=np.int64)
    ip = i ^ xy
    beta_ip = np.where(_v_parity(ip & yz) == 1, -eta, eta)
    return beta_ip * psi[ip]


def apply_pauli_gadget(psi, targs, paulis, theta):
    """Pauli gadget exp(-i theta/2 P) for the Pauli string P on targs.

    Sec. "Pauli gadget" defines U(phi) = exp(i phi P) = cos(phi) 1 +
    i sin(phi) P and the update alpha_i -> cos(phi) alpha_i +
    i sin(phi) beta_{i'} alpha_{i'} (beta, i' as in Sec. "Pauli tensor").
    This library's angle convention is exp(-i theta P / 2), i.e.
    phi = -theta / 2.  With only Z factors this is the phase gadget of
    Sec. "Phase gadget", alpha_i -> exp(i phi s_i) alpha_i.
    """
    psi = np.asarray(psi, dtype=np.complex128)
    nq = _num_qubits(psi)
    _check_qubits(nq, targs)
    phi = -0.5 * theta
    xy, yz, num_y = _pauli_masks(targs, paulis)
    eta = 1j ** num_y
    i = np.arange(1 << nq, dtype=np.int64)
    ip = i ^ xy
    beta_ip = np.where(_v_parity(ip & yz) == 1, -eta, eta)
    return np.cos(phi) * psi + 1j * np.sin(phi) * beta_ip * psi[ip]


def calc_norm(psi):
    """sum_i |alpha_i|^2 (Sec. "Local statevector algorithms": the state
    model)."""
    psi = np.asarray(psi, dtype=np.complex128)
    return float(np.sum(psi.real ** 2 + psi.imag ** 2))


def expec_pauli_sum_statevector(psi, paulis, coeffs):
    """<psi| H |psi> for H = sum_n h_n P_n (Sec. "Pauli string expectation
    value": the statevector form <E> = sum_kl H_lk alpha_k^* alpha_l, for
    which the paper gives no fast algorithm).  paulis is a T x N array of
    codes, row n for term n, column q for qubit q.  Each P_n psi is the Pauli
    tensor of Sec. "Pauli tensor".  Returns a complex number; its real part is
    the expectation value."""
    psi = np.asarray(psi, dtype=np.complex128)
    nq = _num_qubits(psi)
    paulis = np.asarray(paulis).reshape(len(coeffs), nq)
    total = 0j
    for row, h in zip(paulis, coeffs):
        p_psi = apply_pauli_tensor(psi, list(range(nq)), [int(c) for c in row])
        total += h * np.vdot(psi, p_psi)
    return complex(total)


# --------------------------------------------------------------------------
# Density matrices as Choi vectors (Sec. "Distributed density matrix
# algorithms")
# --------------------------------------------------------------------------


def _dm_qubits(rho):
    n2 = _num_qubits(rho)
    if n2 % 2:
        raise ValueError("a Choi vector has an even number of qubits")
    return n2 // 2


def densmatr_from_pure(psi):
    """|psi><psi| as a Choi vector: beta_{j + k 2^N} = psi_j psi_k^*
    (Sec. "State representation", pure-state initialisations)."""
    psi = np.asarray(psi, dtype=np.complex128)
    dim = psi.shape[0]
    out = np.empty(dim * dim, dtype=np.complex128)
    for k in range(dim):
        out[k * dim:(k + 1) * dim] = psi * np.conj(psi[k])
    return out


def densmatr_from_matrix(mat):
    """Choi vector of an explicit matrix rho: beta_{k + l 2^N} = rho[k, l]
    (Sec. "State representation")."""
    mat = np.asarray(mat, dtype=np.complex128)
    dim = mat.shape[0]
    out = np.empty(dim * dim, dtype=np.complex128)
    for l in range(dim):
        out[l * dim:(l + 1) * dim] = mat[:, l]
    return out


def densmatr_to_matrix(rho):
    """Inverse of densmatr_from_matrix."""
    nq = _dm_qubits(rho)
    dim = 1 << nq
    mat = np.empty((dim, dim), dtype=np.complex128)
    for l in range(dim):
        mat[:, l] = rho[l * dim:(l + 1) * dim]
    return mat


def densmatr_apply_ctrl_multi_target(rho, ctrls, targs, mat):
    """U rho U^dagger on a Choi vector: U on (ctrls, targs), then U^* on the
    same qubits shifted by N (Sec. "Unitary gates", Eq. (unitary on a
    vectorised density matrix); controls shift like the targets)."""
    nq = _dm_qubits(rho)
    rho = apply_ctrl_multi_target(rho, ctrls, targs, mat)
    return apply_ctrl_multi_target(rho, [c + nq for c in ctrls], [t + nq for t in targs],
                                   np.conj(np.asarray(mat, dtype=np.complex128)))


def densmatr_apply_diagonal(rho, targs, diag):
    """Diagonal operator D rho D^dagger: D on targs, then D^* on targs + N
    (Sec. "Unitary gates")."""
    nq = _dm_qubits(rho)
    rho = apply_diagonal(rho, targs, diag)
    return apply_diagonal(rho, [t + nq for t in targs], np.conj(np.asarray(diag)))


def densmatr_apply_pauli_gadget(rho, targs, paulis, theta):
    """Pauli gadget on a Choi vector (Algorithm "specific unitaries on density
    matrices"): the gadget on targs, then, because U(theta)^* =
    U((-1)^{#Y+1} theta) for a Pauli string with #Y factors Y, the gadget with
    angle (-1)^{#Y+1} theta on targs + N."""
    nq = _dm_qubits(rho)
    num_y = sum(1 for p in paulis if p == 2)
    rho = apply_pauli_gadget(rho, targs, paulis, theta)
    theta2 = theta * (-1) ** (num_y + 1)
    return apply_pauli_gadget(rho, [t + nq for t in targs], paulis, theta2)


def superoperator(kraus):
    """S = sum_m conj(K_m) (x) K_m (Sec. "Kraus map", Eq. (superoperator from
    a Kraus map)); conj(K) acts on the higher (column, t + N) qubits."""
    kraus = [np.asarray(k, dtype=np.complex128) for k in kraus]
    dim = kraus[0].shape[0]
    sup = np.zeros((dim * dim, dim * dim), dtype=np.complex128)
    for k in kraus:
        sup += np.kron(np.conj(k), k)
    return sup


def densmatr_apply_kraus(rho, targs, kraus):
    """Kraus map rho -> sum_m K_m rho K_m^dagger (Sec. "Kraus map"): the
    superoperator S applied as a dense 2n-target gate on targs u (targs + N),
    matrix bit q on qubit targs[q] and bit n + q on targs[q] + N."""
    nq = _dm_qubits(rho)
    targs = list(targs)
    sup = superoperator(kraus)
    return apply_ctrl_multi_target(rho, [], targs + [t + nq for t in targs], sup)


def densmatr_apply_dephasing(rho, t, p):
    """One-qubit dephasing (Sec. "Dephasing channel"): beta_i -> (1 - 2p)
    beta_i where bit t and bit t + N of i differ; unchanged otherwise."""
    rho = np.array(rho, dtype=np.complex128, copy=True)
    nq = _dm_qubits(rho)
    i = np.arange(rho.shape[0], dtype=np.int64)
    differ = ((i >> t) & 1) != ((i >> (t + nq)) & 1)
    rho[differ] *= 1.0 - 2.0 * p
    return rho


def densmatr_apply_two_qubit_dephasing(rho, t1, t2, p):
    """Two-qubit dephasing (Sec. "Dephasing channel", two-qubit update rule):
    beta_i -> (1 - 4p/3) beta_i if bit t1 differs from bit t1 + N or bit t2
    differs from bit t2 + N."""
    rho = np.array(rho, dtype=np.complex128, copy=True)
    nq = _dm_qubits(rho)
    i = np.arange(rho.shape[0], dtype=np.int64)
    d1 = ((i >> t1) & 1) != ((i >> (t1 + nq)) & 1)
    d2 = ((i >> t2) & 1) != ((i >> (t2 + nq)) & 1)
    rho[d1 | d2] *= 1.0 - 4.0 * p / 3.0
    return rho


def densmatr_apply_depolarising(rho, t, p):
    """One-qubit depolarising (Sec. "Depolarising channel", Eq. (one-qubit
    depolarising amplitude update)): where bits t and t + N agree,
    beta_i -> (1 - 2p/3) beta_i + (2p/3) beta_{i with both bits flipped};
    where they differ, beta_i -> (1 - 4p/3) beta_i."""
    rho = np.asarray(rho, dtype=np.complex128)
    nq = _dm_qubits(rho)
    i = np.arange(rho.shape[0], dtype=np.int64)
    same = ((i >> t) & 1) == ((i >> (t + nq)) & 1)
    partner = i ^ ((1 << t) | (1 << (t + nq)))
    out = np.where(same,
                   (1.0 - 2.0 * p / 3.0) * rho + (2.0 * p / 3.0) * rho[partner],
                   (1.0 - 4.0 * p / 3.0) * rho)
    return out


def densmatr_apply_two_qubit_depolarising(rho, t1, t2, p):
    """Two-qubit depolarising (Sec. "Depolarising channel", Eq. (two-qubit
    depolarising Choi amplitude update)): where bits t1 = t1 + N and
    t2 = t2 + N, beta_i -> (1 - 4p/5) beta_i + (4p/15)(beta_{i flip t1,t1+N}
    + beta_{i flip t2,t2+N} + beta_{i flip all four}); otherwise
    beta_i -> (1 - 16p/15) beta_i.  This follows the equation; the
    coefficients in the paper's listing of this channel disagree with it."""
    rho = np.asarray(rho, dtype=np.complex128)
    nq = _dm_qubits(rho)
    i = np.arange(rho.shape[0], dtype=np.int64)
    same = ((((i >> t1) & 1) == ((i >> (t1 + nq)) & 1))
            & (((i >> t2) & 1) == ((i >> (t2 + nq)) & 1)))
    f1 = (1 << t1) | (1 << (t1 + nq))
    f2 = (1 << t2) | (1 << (t2 + nq))
    mixed = ((1.0 - 4.0 * p / 5.0) * rho
             + (4.0 * p / 15.0) * (rho[i ^ f1] + rho[i ^ f2] + rho[i ^ f1 ^ f2]))
    return np.where(same, mixed, (1.0 - 16.0 * p / 15.0) * rho)


def densmatr_apply_damping(rho, t, p):
    """Amplitude damping (Sec. "Damping channel", Eq. (damping amplitude
    update)): bits (t, t + N) = (0, 0): beta_i + p beta_{i flip both};
    bits differ: sqrt(1 - p) beta_i; bits (1, 1): (1 - p) beta_i."""
    rho = np.asarray(rho, dtype=np.complex128)
    nq = _dm_qubits(rho)
    i = np.arange(rho.shape[0], dtype=np.int64)
    b_lo = (i >> t) & 1
    b_hi = (i >> (t + nq)) & 1
    partner = i ^ ((1 << t) | (1 << (t + nq)))
    out = np.where((b_lo == 0) & (b_hi == 0), rho + p * rho[partner],
                   np.where(b_lo != b_hi, np.sqrt(1.0 - p) * rho, (1.0 - p) * rho))
    return out


def densmatr_apply_pauli_channel(rho, t, px, py, pz):
    """One-qubit Pauli channel rho -> (1 - px - py - pz) rho + px X rho X +
    py Y rho Y + pz Z rho Z on qubit t: the general form of the depolarising
    channel (Sec. "Depolarising channel", which notes the extension).  Each
    sigma rho sigma is the unitary sigma applied to the Choi vector (Sec.
    "Unitary gates": sigma on t, conj(sigma) on t + N)."""
    rho = np.asarray(rho, dtype=np.complex128)
    sx = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    sy = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
    sz = np.array([[1, 0], [0, -1]], dtype=np.complex128)
    out = (1.0 - px - py - pz) * rho
    for p, sig in ((px, sx), (py, sy), (pz, sz)):
        out = out + p * densmatr_apply_ctrl_multi_target(rho, [], [t], sig)
    return out


def partial_trace(rho, targs):
    """Partial trace over targs (Sec. "Partial trace", Eqs. (reduced amplitude
    definition) and (index function)): beta'_i = sum_v beta_{g(i, v)}, where
    g(i, v) interweaves the bits of (v << n) | v into positions
    targs u (targs + N) and the bits of i, in order, into the remaining
    positions.  The result is the Choi vector of N - n qubits; the kept qubits
    keep their relative order."""
    rho = np.asarray(rho, dtype=np.complex128)
    nq = _dm_qubits(rho)
    targs = list(targs)
    _check_qubits(nq, targs)
    n = len(targs)
    m = nq - n
    traced_positions = targs + [t + nq for t in targs]
    kept_positions = sorted(set(range(2 * nq)) - set(traced_positions))
    out = np.zeros(1 << (2 * m), dtype=np.complex128)
    i = np.arange(1 << (2 * m), dtype=np.int64)
    base = np.zeros_like(i)
    for q, pos in enumerate(kept_positions):
        base |= ((i >> q) & 1) << pos
    for v in range(1 << n):
        vv = (v << n) | v
        off = set_bits(0, traced_positions, vv)
        out += rho[base | off]
    return out


def pauli_tensor_elem(sigma_row, i, nq):
    """Element <row bits| sigma_{N-1} ... sigma_0 |col bits> of a Pauli tensor
    at Choi index i: column bit q is i_[q], row bit q is i_[q + N]
    (Algorithm "Pauli string expectation value": pauliTensorElem).  Vectorised
    over an int64 array i."""
    mats = [np.array([[1, 0], [0, 1]], dtype=np.complex128),
            np.array([[0, 1], [1, 0]], dtype=np.complex128),
            np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
            np.array([[1, 0], [0, -1]], dtype=np.complex128)]
    v = np.ones(i.shape, dtype=np.complex128)
    for q in range(nq):
        b_c = (i >> q) & 1
        b_r = (i >> (q + nq)) & 1
        v = v * mats[int(sigma_row[q])][b_r, b_c]
    return v


def expec_pauli_sum_densmatr(rho, paulis, coeffs):
    """Tr(H rho) for H = sum_n h_n P_n (Sec. "Pauli string expectation value",
    Eq. (density expectation sum)): sum_i H_i beta_i with
    H_i = sum_n h_n pauliTensorElem(sigma^(n), i).  paulis is T x N, row n for
    term n, column q for qubit q.  Returns a complex number; its real part is
    the expectation value (the imaginary part vanishes for Hermitian rho)."""
    rho = np.asarray(rho, dtype=np.complex128)
    nq = _dm_qubits(rho)
    paulis = np.asarray(paulis).reshape(len(coeffs), nq)
    i = np.arange(rho.shape[0], dtype=np.int64)
    h_i = np.zeros(rho.shape[0], dtype=np.complex128)
    for row, h in zip(paulis, coeffs):
        h_i += h * pauli_tensor_elem(row, i, nq)
    return complex(np.sum(h_i * rho))


def calc_trace(rho):
    """Tr rho = sum_j beta_{j (2^N + 1)} (Sec. "Pauli string expectation
    value")."""
    rho = np.asarray(rho, dtype=np.complex128)
    nq = _dm_qubits(rho)
    dim = 1 << nq
    return complex(np.sum(rho[np.arange(dim) * (dim + 1)]))


# --------------------------------------------------------------------------
# Circuit runner: applies a list of operation records (the format produced by
# the seeded workload generators) one by one.
# --------------------------------------------------------------------------


def run_ops(state, ops, is_density):
    """Apply each record of ops in order and return the final state."""
    s = np.array(state, dtype=np.complex128, copy=True)
    for op in ops:
        kind = op["op"]
        if kind == "unitary":
            f = densmatr_apply_ctrl_multi_target if is_density else apply_ctrl_multi_target
            s = f(s, op["ctrls"], op["targs"], op["mat"])
        elif kind == "diagonal":
            f = densmatr_apply_diagonal if is_density else apply_diagonal
            s = f(s, op["targs"], op["diag"])
        elif kind == "gadget":
            f = densmatr_apply_pauli_gadget if is_density else apply_pauli_gadget
            s = f(s, op["targs"], op["paulis"], op["theta"])
        elif kind == "kraus":
            s = densmatr_apply_kraus(s, op["targs"], op["kraus"])
        elif kind == "dephasing":
            s = densmatr_apply_dephasing(s, op["targs"][0], op["p"])
        elif kind == "dephasing2":
            s = densmatr_apply_two_qubit_dephasing(s, op["targs"][0], op["targs"][1], op["p"])
        elif kind == "depolarising":
            s = densmatr_apply_depolarising(s, op["targs"][0], op["p"])
        elif kind == "depolarising2":
            s = densmatr_apply_two_qubit_depolarising(s, op["targs"][0], op["targs"][1], op["p"])
        elif kind == "damping":
            s = densmatr_apply_damping(s, op["targs"][0], op["p"])
        elif kind == "pauli_channel":
            s = densmatr_apply_pauli_channel(s, op["targs"][0], *op["probs"])
        elif kind == "swap":
            f = densmatr_apply_swap if is_density else apply_swap
            s = f(s, op["targs"][0], op["targs"][1])
        else:
            raise ValueError("unknown op " + kind)
    return s


# --------------------------------------------------------------------------
# Single-amplitude evaluation, for states too large to process whole: each
# function returns the new amplitudes at the output indices `out_idx`, given
# `get(indices)` that returns the OLD amplitudes at any indices.  Same
# definitions as above, evaluated one output at a time.
# --------------------------------------------------------------------------


def sample_ctrl_multi_target(get, ctrls, targs, mat, out_idx):
    """New amplitudes at out_idx after the many-control many-target gate
    (Sec. "Many-target gate", Eq. (local many-target amplitude update); Sec.
    "Many-control one-target gate", Eq. (control condition))."""
    mat = np.asarray(mat, dtype=np.complex128)
    n = len(targs)
    cmask = get_bit_mask(ctrls)
    tmask = get_bit_mask(targs)
    out = np.empty(len(out_idx), dtype=np.complex128)
    for o, i in enumerate(int(x) for x in out_idx):
        if (i & cmask) != cmask:
            out[o] = get(np.array([i]))[0]
            continue
        j = sum(get_bit(i, t) << q for q, t in enumerate(targs))
        base = i & ~tmask
        partners = np.array([set_bits(base, targs, l) for l in range(1 << n)], dtype=np.int64)
        out[o] = np.dot(mat[j, :], get(partners))
    return out


def sample_diagonal(get, targs, diag, out_idx):
    """New amplitudes at out_idx after the diagonal operator."""
    diag = np.asarray(diag, dtype=np.complex128)
    idx = np.asarray(out_idx, dtype=np.int64)
    j = np.zeros_like(idx)
    for q, t in enumerate(targs):
        j |= ((idx >> t) & 1) << q
    return diag[j] * get(idx)


def sample_pauli_gadget(get, targs, paulis, theta, out_idx):
    """New amplitudes at out_idx after exp(-i theta/2 P) (Sec. "Pauli
    gadget")."""
    phi = -0.5 * theta
    xy, yz, num_y = _pauli_masks(targs, paulis)
    eta = 1j ** num_y
    idx = np.asarray(out_idx, dtype=np.int64)
    ip = idx ^ xy
    beta = np.where(_v_parity(ip & yz) == 1, -eta, eta)
    return np.cos(phi) * get(idx) + 1j * np.sin(phi) * beta * get(ip)


def sample_swap(get, t1, t2, out_idx):
    """New amplitudes at out_idx after SWAP of qubits t1, t2 (Sec. "Swap
    gate"): alpha_{i with both bits flipped} where the two bits differ."""
    idx = np.asarray(out_idx, dtype=np.int64)
    differ = ((idx >> t1) & 1) != ((idx >> t2) & 1)
    src = np.where(differ, idx ^ ((1 << t1) | (1 << t2)), idx)
    return get(src)


def _sample_bits(idx, t, nq):
    """Bits t and t + N of each Choi index in idx (column and row bit of qubit t)."""
    return (idx >> t) & 1, (idx >> (t + nq)) & 1


def sample_densmatr_dephasing(get, nq, t, p, out_idx):
    """New Choi amplitudes at out_idx after one-qubit dephasing (Sec.
    "Dephasing channel"): scaled by (1 - 2p) where bits t and t + N differ."""
    idx = np.asarray(out_idx, dtype=np.int64)
    lo, hi = _sample_bits(idx, t, nq)
    return np.where(lo != hi, 1.0 - 2.0 * p, 1.0) * get(idx)


def sample_densmatr_two_qubit_dephasing(get, nq, t1, t2, p, out_idx):
    """Two-qubit dephasing (Sec. "Dephasing channel"): scaled by (1 - 4p/3)
    where bits t1, t1 + N or bits t2, t2 + N differ."""
    idx = np.asarray(out_idx, dtype=np.int64)
    a_lo, a_hi = _sample_bits(idx, t1, nq)
    b_lo, b_hi = _sample_bits(idx, t2, nq)
    return np.where((a_lo != a_hi) | (b_lo != b_hi), 1.0 - 4.0 * p / 3.0, 1.0) * get(idx)


def sample_densmatr_depolarising(get, nq, t, p, out_idx):
    """One-qubit depolarising (Sec. "Depolarising channel"): where bits t and
    t + N agree, (1 - 2p/3) beta_i + (2p/3) beta_{i with both flipped}; where
    they differ, (1 - 4p/3) beta_i."""
    idx = np.asarray(out_idx, dtype=np.int64)
    lo, hi = _sample_bits(idx, t, nq)
    partner = idx ^ ((1 << t) | (1 << (t + nq)))
    same = (1.0 - 2.0 * p / 3.0) * get(idx) + (2.0 * p / 3.0) * get(partner)
    return np.where(lo == hi, same, (1.0 - 4.0 * p / 3.0) * get(idx))


def sample_densmatr_two_qubit_depolarising(get, nq, t1, t2, p, out_idx):
    """Two-qubit depolarising (Sec. "Depolarising channel", the equation):
    where both bit pairs agree, (1 - 4p/5) beta_i + (4p/15) times the sum of
    the three partners with one or both pairs flipped; otherwise
    (1 - 16p/15) beta_i."""
    idx = np.asarray(out_idx, dtype=np.int64)
    a_lo, a_hi = _sample_bits(idx, t1, nq)
    b_lo, b_hi = _sample_bits(idx, t2, nq)
    f1 = (1 << t1) | (1 << (t1 + nq))
    f2 = (1 << t2) | (1 << (t2 + nq))
    mixed = (1.0 - 4.0 * p / 5.0) * get(idx) + (4.0 * p / 15.0) * (get(idx ^ f1) + get(idx ^ f2) + get(idx ^ f1 ^ f2))
    return np.where((a_lo == a_hi) & (b_lo == b_hi), mixed, (1.0 - 16.0 * p / 15.0) * get(idx))


def sample_densmatr_damping(get, nq, t, p, out_idx):
    """Amplitude damping (Sec. "Damping channel"): bits (t, t + N) = (0, 0):
    beta_i + p beta_{both flipped}; bits differ: sqrt(1 - p) beta_i; bits
    (1, 1): (1 - p) beta_i."""
    idx = np.asarray(out_idx, dtype=np.int64)
    lo, hi = _sample_bits(idx, t, nq)
    partner = idx ^ ((1 << t) | (1 << (t + nq)))
    return np.where((lo == 0) & (hi == 0), get(idx) + p * get(partner),
                    np.where(lo != hi, np.sqrt(1.0 - p) * get(idx), (1.0 - p) * get(idx)))


def sample_densmatr_pauli_channel(get, nq, t, px, py, pz, out_idx):
    """One-qubit Pauli channel (1 - px - py - pz) rho + px X rho X + py Y rho Y
    + pz Z rho Z, one output at a time: sigma rho sigma^dagger has Choi
    amplitudes sigma[r', r] conj(sigma[c', c]) beta_{partner} with
    (c, r) = bits (t, t + N) of i and the partner's bits (c', r') fixed by
    sigma's single non-zero entry per row."""
    idx = np.asarray(out_idx, dtype=np.int64)
    c, r = _sample_bits(idx, t, nq)
    out = (1.0 - px - py - pz) * get(idx)
    both = (1 << t) | (1 << (t + nq))
    # X: <r|X|r'> = 1 for r' = 1 - r, same for the column
    out = out + px * get(idx ^ both)
    # Y: Y[r, 1-r] = -i (r = 0) or i (r = 1); conj(Y[c, 1-c]) = i (c = 0) or -i (c = 1)
    yr = np.where(r == 0, -1j, 1j)
    yc = np.where(c == 0, 1j, -1j)
    out = out + py * yr * yc * get(idx ^ both)
    # Z: Z[r, r] Z[c, c] = (-1)^(r + c)
    out = out + pz * np.where(r == c, 1.0, -1.0) * get(idx)
    return out
