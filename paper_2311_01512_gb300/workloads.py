"""Seeded synthetic inputs: random states, Haar unitaries, Kraus channels,
Pauli strings and random circuits.

This module only draws inputs.  It holds none of the simulation arithmetic and
is shared by the CUDA path's tests and benchmark and by the oracle-side tests,
so that both sides see identical inputs.  It imports numpy only.

Operation records are plain dicts:

* ``{"op": "unitary", "ctrls": [...], "targs": [...], "mat": (2^n, 2^n) complex}``
* ``{"op": "diagonal", "targs": [...], "diag": (2^n,) complex}``
* ``{"op": "gadget", "targs": [...], "paulis": [...], "theta": float}``
  (exp(-i theta P / 2), Pauli codes 0 = I, 1 = X, 2 = Y, 3 = Z)
* ``{"op": "kraus", "targs": [...], "kraus": [(2^n, 2^n) complex, ...]}``
* ``{"op": "dephasing" | "depolarising" | "damping", "targs": [t], "p": float}``
* ``{"op": "dephasing2" | "depolarising2", "targs": [t1, t2], "p": float}``
"""

import numpy as np

SEED_BASE = 2311015120


def rng_for(tag, seed=SEED_BASE):
    """Independent generator per purpose (state, circuit, ...)."""
    tag_code = sum((i + 1) * ord(c) for i, c in enumerate(tag))
    return np.random.default_rng([seed, tag_code])


def haar_unitary(dim, rng):
    """Haar-random unitary: QR of a complex Ginibre matrix with the phases of
    R's diagonal moved into Q (Mezzadri, "How to generate random matrices from
    the classical compact groups", 2007)."""
    z = (rng.standard_normal((dim, dim)) + 1j * rng.standard_normal((dim, dim))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r)
    return q * (d / np.abs(d))[None, :]


def haar_kraus(num_qubits, num_ops, rng):
    """Random channel of num_ops Kraus operators on num_qubits qubits from a
    Haar isometry V : C^d -> C^{num_ops d} (the first d columns of a Haar
    unitary), cut into num_ops blocks of d rows.  sum_m K_m^dag K_m = 1."""
    d = 1 << num_qubits
    u = haar_unitary(d * num_ops, rng)
    v = u[:, :d]
    return [np.ascontiguousarray(v[m * d:(m + 1) * d, :]) for m in range(num_ops)]


def random_statevector(num_qubits, rng, dtype=np.complex128):
    """Normalised vector of i.i.d. complex Gaussian amplitudes."""
    dim = 1 << num_qubits
    psi = rng.standard_normal(dim) + 1j * rng.standard_normal(dim)
    psi /= np.sqrt(np.sum(psi.real ** 2 + psi.imag ** 2))
    return psi.astype(dtype)


def random_mixture_weights(rank, rng):
    w = rng.random(rank)
    return w / w.sum()


def random_pauli_string(num_qubits, min_weight, max_weight, rng):
    """Weight w uniform in [min_weight, max_weight]; w distinct qubits chosen
    uniformly; each factor uniform over {X, Y, Z}.  Returns (targs, paulis)."""
    w = int(rng.integers(min_weight, max_weight + 1))
    targs = [int(x) for x in rng.choice(num_qubits, size=w, replace=False)]
    paulis = [int(x) for x in rng.integers(1, 4, size=w)]
    return targs, paulis


def random_pauli_sum(num_qubits, num_terms, rng, coeff="normal"):
    """num_terms random Pauli strings over all num_qubits qubits (each
    factor uniform over {I, X, Y, Z}) and real coefficients."""
    paulis = rng.integers(0, 4, size=(num_terms, num_qubits)).astype(np.int32)
    if coeff == "normal":
        coeffs = rng.standard_normal(num_terms)
    else:
        coeffs = rng.uniform(-1.0, 1.0, size=num_terms)
    return paulis, coeffs


def _distinct(num_qubits, count, rng):
    return [int(x) for x in rng.choice(num_qubits, size=count, replace=False)]


def _unitary_op(num_qubits, rng, min_targs, max_targs, max_ctrls):
    n = int(rng.integers(min_targs, max_targs + 1))
    s = int(rng.integers(0, max_ctrls + 1))
    s = min(s, num_qubits - n)
    qs = _distinct(num_qubits, n + s, rng)
    return {"op": "unitary", "targs": qs[:n], "ctrls": qs[n:], "mat": haar_unitary(1 << n, rng)}


def _gadget_op(num_qubits, rng, min_w, max_w):
    targs, paulis = random_pauli_string(num_qubits, min_w, min(max_w, num_qubits), rng)
    return {"op": "gadget", "targs": targs, "paulis": paulis,
            "theta": float(rng.uniform(0.0, 2.0 * np.pi))}


def _diag_op(num_qubits, rng, min_targs, max_targs):
    n = int(rng.integers(min_targs, max_targs + 1))
    targs = _distinct(num_qubits, n, rng)
    phases = rng.uniform(0.0, 2.0 * np.pi, size=1 << n)
    return {"op": "diagonal", "targs": targs, "diag": np.exp(1j * phases)}


def statevector_circuit(num_qubits, num_ops, rng, max_targs=5, max_ctrls=5, max_gadget_weight=None):
    """Circuit of the 30-qubit statevector workload: one-qubit Haar unitaries on
    uniform qubits; Haar unitaries on 2..max_targs targets with
    0..max_ctrls controls; 1..3-qubit diagonal phase gates; Pauli gadgets of
    weight 1..num_qubits.  The four kinds are drawn with equal probability."""
    if max_gadget_weight is None:
        max_gadget_weight = num_qubits
    ops = []
    for _ in range(num_ops):
        kind = int(rng.integers(0, 4))
        if kind == 0:
            ops.append(_unitary_op(num_qubits, rng, 1, 1, 0))
        elif kind == 1:
            ops.append(_unitary_op(num_qubits, rng, 2, max_targs, max_ctrls))
        elif kind == 2:
            ops.append(_diag_op(num_qubits, rng, 1, 3))
        else:
            ops.append(_gadget_op(num_qubits, rng, 1, max_gadget_weight))
    return ops


def unitary_circuit(num_qubits, num_ops, rng):
    """Unitary-only circuit: one-qubit Haar unitaries; 1..2-target Haar
    unitaries with 0..3 controls; Pauli gadgets of weight 1..6 (equal
    probability)."""
    ops = []
    for _ in range(num_ops):
        kind = int(rng.integers(0, 3))
        if kind == 0:
            ops.append(_unitary_op(num_qubits, rng, 1, 1, 0))
        elif kind == 1:
            ops.append(_unitary_op(num_qubits, rng, 1, 2, 3))
        else:
            ops.append(_gadget_op(num_qubits, rng, 1, 6))
    return ops


def small_densmatr_circuit(num_qubits, num_ops, rng):
    """Circuit of the 6-qubit density-matrix workload: one-qubit Haar unitaries;
    1..2-target Haar unitaries with 0..3 controls; Pauli gadgets (weight 1..6,
    theta ~ U[0, 2 pi)); one-qubit depolarising (p ~ U[0, 0.1]); amplitude
    damping (p ~ U[0, 0.1]); two-qubit channels of 4 Kraus operators from a
    Haar isometry.  The six kinds are drawn with equal probability."""
    ops = []
    for _ in range(num_ops):
        kind = int(rng.integers(0, 6))
        if kind == 0:
            ops.append(_unitary_op(num_qubits, rng, 1, 1, 0))
        elif kind == 1:
            ops.append(_unitary_op(num_qubits, rng, 1, 2, 3))
        elif kind == 2:
            ops.append(_gadget_op(num_qubits, rng, 1, 6))
        elif kind == 3:
            ops.append({"op": "depolarising", "targs": _distinct(num_qubits, 1, rng),
                        "p": float(rng.uniform(0.0, 0.1))})
        elif kind == 4:
            ops.append({"op": "damping", "targs": _distinct(num_qubits, 1, rng),
                        "p": float(rng.uniform(0.0, 0.1))})
        else:
            ops.append({"op": "kraus", "targs": _distinct(num_qubits, 2, rng),
                        "kraus": haar_kraus(2, 4, rng)})
    return ops


def large_densmatr_circuit(num_qubits, num_ops, rng):
    """Circuit of the 15-qubit density-matrix workload: Haar unitaries on 1..3
    targets with 0..3 controls; one- and two-qubit depolarising and
    dephasing; amplitude damping (all p ~ U[0, 0.1]); two-qubit 4-Kraus
    channels.  The seven kinds are drawn with equal probability."""
    ops = []
    for _ in range(num_ops):
        kind = int(rng.integers(0, 7))
        p = float(rng.uniform(0.0, 0.1))
        if kind == 0:
            ops.append(_unitary_op(num_qubits, rng, 1, 3, 3))
        elif kind == 1:
            ops.append({"op": "depolarising", "targs": _distinct(num_qubits, 1, rng), "p": p})
        elif kind == 2:
            ops.append({"op": "depolarising2", "targs": _distinct(num_qubits, 2, rng), "p": p})
        elif kind == 3:
            ops.append({"op": "dephasing", "targs": _distinct(num_qubits, 1, rng), "p": p})
        elif kind == 4:
            ops.append({"op": "dephasing2", "targs": _distinct(num_qubits, 2, rng), "p": p})
        elif kind == 5:
            ops.append({"op": "damping", "targs": _distinct(num_qubits, 1, rng), "p": p})
        else:
            ops.append({"op": "kraus", "targs": _distinct(num_qubits, 2, rng),
                        "kraus": haar_kraus(2, 4, rng)})
    return ops


def random_mixed_state_vectors(num_qubits, rank, rng):
    """rank normalised Gaussian pure states and mixture weights; the density
    matrix is sum_m w_m |psi_m><psi_m|."""
    states = [random_statevector(num_qubits, rng) for _ in range(rank)]
    return states, random_mixture_weights(rank, rng)
