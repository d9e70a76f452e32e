"""The persistent batched engine (qs_batch_*): every state of a batch with its
own random circuit, run in one recorded launch, against the CPU oracle state
by state (complex128 in double-float: 1e-12 per 1000 gates; complex64: 1 - F
<= 1e-6).  Sizes include states too large for shared memory, so both the
shared-memory path and the tiled path (segments of operations applied tile by
tile, with controls, diagonal targets and gadget phase qubits both inside and
outside the tile) run, and so does the global-memory path of an operation
that pairs more qubits than a tile holds."""

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
def test_batch_matches_oracle(qs, prec):
    import torch
    rng = wl.rng_for("batch-test-%d" % prec)
    sizes = [int(x) for x in rng.integers(3, 14, size=40)] + [15, 16, 17]
    batch = qs.Batch(sizes, prec=prec)
    circuits = []
    for s, nq in enumerate(sizes):
        ops = wl.unitary_circuit(nq, int(rng.integers(10, 60)), rng)
        for k in range(0, len(ops), 5):             # diagonals on 1..3 qubits
            n = int(rng.integers(1, min(3, nq) + 1))
            targs = [int(x) for x in rng.choice(nq, n, replace=False)]
            ops.insert(k, {"op": "diagonal", "targs": targs,
                           "diag": np.exp(1j * rng.uniform(0, 2 * np.pi, 1 << n))})
        if nq >= 15:                                 # X/Y on every qubit: more than a tile
            ops.insert(len(ops) // 2, {"op": "gadget", "targs": list(range(nq)),
                                       "paulis": [int(x) for x in rng.integers(1, 3, nq)], "theta": 0.7})
        for op in ops:
            batch.add(s, op)
        circuits.append(ops)
    batch.compile(autotune=True)
    info = batch.info()
    assert info["smem_qubits"] < 17            # the largest states take the global path
    dtype = np.complex128 if prec == 1 else np.complex64
    inits = [wl.random_statevector(nq, rng) for nq in sizes]
    for s, psi in enumerate(inits):
        batch.view(s).copy_(torch.from_numpy(psi.astype(dtype)))
    batch.run()
    batch.run()                                 # the recorded launch replays
    torch.cuda.synchronize()
    for s, (psi, ops) in enumerate(zip(inits, circuits)):
        want = orc.run_ops(orc.run_ops(psi, ops, False), ops, False)
        got = batch.view(s).cpu().numpy().astype(np.complex128)
        if prec == 1:
            assert float(np.max(np.abs(got - want))) <= 1e-12, s
        else:
            fid = abs(np.vdot(want, got)) ** 2 / (np.vdot(got, got).real * np.vdot(want, want).real)
            assert 1.0 - fid <= 1e-6, (s, 1.0 - fid)


def test_batch_validation(qs):
    batch = qs.Batch([4, 5])
    with pytest.raises(qs.QSError):
        batch.add(0, {"op": "unitary", "ctrls": [], "targs": [0, 1, 2], "mat": np.eye(8)})
    with pytest.raises(qs.QSError):
        batch.add(1, {"op": "unitary", "ctrls": [], "targs": [5], "mat": np.eye(2)})
    with pytest.raises(qs.QSError):
        batch.add(2, {"op": "unitary", "ctrls": [], "targs": [0], "mat": np.eye(2)})


@pytest.mark.parametrize("prec", [1, 0])
def test_batch_density_matrices(qs, prec):
    """Density matrices in a batch (Choi vectors of 6 to 16 storage qubits,
    the largest beyond shared memory) next to statevectors: unitaries with
    controls, diagonals and gadgets as U on t and U* on t + N, Kraus maps and
    every channel as superoperator passes, against the oracle."""
    import torch
    rng = wl.rng_for("batch-dm-%d" % prec)
    sizes = [3, 4, 5, 6, 7, 8, 5, 6]
    dens = [True] * 6 + [False] * 2
    batch = qs.Batch(sizes, prec=prec, density=dens)
    circuits, inits = [], []
    for s, (nq, d) in enumerate(zip(sizes, dens)):
        if d:
            ops = wl.small_densmatr_circuit(nq, 30, rng)
            ops += [{"op": "dephasing", "targs": [nq - 1], "p": 0.06},
                    {"op": "dephasing2", "targs": [0, nq - 1], "p": 0.05},
                    {"op": "depolarising2", "targs": [nq - 2, 0], "p": 0.04},
                    {"op": "pauli_channel", "targs": [1], "probs": (0.03, 0.02, 0.01)},
                    {"op": "diagonal", "targs": [nq - 1, 0],
                     "diag": np.exp(1j * rng.uniform(0, 2 * np.pi, 4))}]
            states, w = wl.random_mixed_state_vectors(nq, 2, rng)
            init = sum(wi * orc.densmatr_from_pure(v) for wi, v in zip(w, states))
        else:
            ops = wl.unitary_circuit(nq, 30, rng)
            init = wl.random_statevector(nq, rng)
        for op in ops:
            batch.add(s, op)
        circuits.append(ops)
        inits.append(init)
    with pytest.raises(qs.QSError):
        batch.add(6, {"op": "damping", "targs": [0], "p": 0.1})      # a statevector takes no channel
    batch.compile(autotune=True)
    dtype = np.complex128 if prec == 1 else np.complex64
    for s, init in enumerate(inits):
        batch.view(s).copy_(torch.from_numpy(init.astype(dtype)))
    batch.run()
    batch.run()
    torch.cuda.synchronize()
    for s, (init, ops, d) in enumerate(zip(inits, circuits, dens)):
        want = orc.run_ops(orc.run_ops(init, ops, d), ops, d)
        got = batch.view(s).cpu().numpy().astype(np.complex128)
        err = float(np.max(np.abs(got - want)))
        assert err <= (1e-12 if prec == 1 else 2e-5), (s, err)


def test_batch_edge_cases(qs):
    """States with no operations (left unchanged, in shared memory and tiled),
    one-qubit states, and a one-state batch."""
    import torch
    rng = wl.rng_for("batch-edge")
    sizes = [1, 2, 11, 15, 15]
    nops = [3, 0, 5, 0, 12]
    batch = qs.Batch(sizes, prec=1)
    circuits = []
    for s, (nq, k) in enumerate(zip(sizes, nops)):
        ops = wl.unitary_circuit(nq, k, rng) if k else []
        for op in ops:
            batch.add(s, op)
        circuits.append(ops)
    batch.compile(autotune=False)
    inits = [wl.random_statevector(nq, rng) for nq in sizes]
    for s, psi in enumerate(inits):
        batch.view(s).copy_(torch.from_numpy(psi))
    batch.run()
    torch.cuda.synchronize()
    for s, (psi, ops) in enumerate(zip(inits, circuits)):
        got = batch.view(s).cpu().numpy()
        want = orc.run_ops(psi, ops, False) if ops else psi
        assert float(np.max(np.abs(got - want))) <= 1e-13, s
    one = qs.Batch([3], prec=0)
    op = {"op": "unitary", "ctrls": [2], "targs": [0, 1], "mat": wl.haar_unitary(4, rng)}
    one.add(0, op)
    one.compile(autotune=True)
    psi = wl.random_statevector(3, rng)
    one.view(0).copy_(torch.from_numpy(psi.astype(np.complex64)))
    one.run()
    torch.cuda.synchronize()
    want = orc.run_ops(psi, [op], False)
    assert float(np.max(np.abs(one.view(0).cpu().numpy() - want))) <= 1e-6
