"""CUDA path vs the oracle at sizes where every grid-stride loop of the
streaming, channel and reduction kernels runs more than once per thread.

The streaming grids hold at most 152 x 256 blocks of 256 threads (about
2^23.2), the reduction grids 1216 (expectation values) or 4864 (norm) blocks
of 256.  So:
* a 13-qubit density matrix (26-qubit Choi vector, 1 GiB) gives one-qubit
  channels 2^24 groups, the pure-state initialisation 2^26 elements and a
  partial trace of one qubit 2^24 outputs: compared with the whole-vector
  oracle, in block fixed point and in double-float;
* a 14-qubit density matrix (28-qubit Choi vector, 4 GiB) gives two-qubit
  channels 2^24 groups: compared at sampled outputs with the oracle's
  single-output forms of the same equations;
* a 10-qubit density matrix with 320 Pauli terms gives the expectation kernel
  320 2^10 > 1216 x 256 work items;
* a 22-qubit statevector gives the statevector expectation kernels 4096
  tiles of 1024 amplitudes (1216 blocks) and 2^15 warp tiles (9728 warps).
Tolerances are those of the small-size parity tests (tests/test_gpu_parity.py).
"""

import numpy as np
import pytest

from oracle import qsim_oracle as orc
from paper_2311_01512_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

# per-operation max |delta amp| and scalar tolerances by arithmetic
ATOL = {"fx": 1e-14, "df": 1e-13}
STOL = {"fx": 1e-14, "df": 1e-12}


@pytest.fixture(scope="module")
def qs():
    from paper_2311_01512_gb300 import qs as mod
    return mod


def arith_code(qs, arith):
    return qs.QS_ARITH_FX if arith == "fx" else qs.QS_ARITH_DF


def maxdiff(got, want):
    return float(np.max(np.abs(np.asarray(got, dtype=np.complex128) - want)))


@pytest.mark.parametrize("arith", ["fx", "df"])
def test_statevector_expectation_22_qubits(qs, arith):
    rng = np.random.default_rng(2222)
    nq = 22
    psi = wl.random_statevector(nq, rng)
    st = qs.State(nq, density=False, prec=qs.QS_C128)
    qs.qs_set_arithmetic(st.handle, arith_code(qs, arith))
    st.set_amps(psi)
    paulis, coeffs = wl.random_pauli_sum(nq, 24, rng)
    # flip masks with their highest bit below and above a 1024-amplitude tile
    extra = np.zeros((4, nq), dtype=np.int32)
    extra[0, 3] = 1
    extra[1, 9] = 2
    extra[2, 15] = 1
    extra[3, nq - 1] = 2
    extra[3, 0] = 3
    paulis = np.concatenate([paulis, extra])
    coeffs = np.concatenate([coeffs, rng.standard_normal(4)])
    got = qs.qs_expec_pauli_sum(st.handle, paulis, coeffs)
    want = orc.expec_pauli_sum_statevector(psi, paulis, coeffs)
    assert abs(got - want) < STOL[arith] * np.abs(coeffs).sum(), (got, want)
    # 40 I/Z strings: the warp Walsh-Hadamard kernel
    zs = np.where(rng.random((40, nq)) < 0.4, 3, 0).astype(np.int32)
    zs[0, :] = 0
    zs[1, nq - 1] = 3
    hz = rng.standard_normal(40)
    got_z = qs.qs_expec_pauli_sum(st.handle, zs, hz)
    want_z = orc.expec_pauli_sum_statevector(psi, zs, hz)
    assert abs(got_z - want_z) < STOL[arith] * np.abs(hz).sum(), (got_z, want_z)
    norm = qs.qs_calc_norm_or_trace(st.handle)
    assert abs(norm - orc.calc_norm(psi)) < STOL[arith]
    st.close()


def test_densmatr_13_qubits_whole_vector(qs):
    """Initialisation from a rank-2 mixture, one-qubit channels, a Kraus map
    and a controlled two-target unitary on a 26-qubit Choi vector, each
    compared with the oracle over the whole vector; then a partial trace of
    one qubit (2^24 outputs) and the trace."""
    rng = np.random.default_rng(1313)
    nq = 13
    states = [wl.random_statevector(nq, rng) for _ in range(2)]
    w = [0.6, 0.4]
    want = sum(wi * orc.densmatr_from_pure(s) for wi, s in zip(w, states))
    dms = {}
    for arith in ("fx", "df"):
        dm = qs.State(nq, density=True, prec=qs.QS_C128)
        qs.qs_set_arithmetic(dm.handle, arith_code(qs, arith))
        for m, (s, wi) in enumerate(zip(states, w)):
            sv = qs.State(nq, density=False, prec=qs.QS_C128)
            qs.qs_set_arithmetic(sv.handle, arith_code(qs, arith))
            sv.set_amps(s)
            qs.qs_init_pure_densmatr(dm.handle, sv.handle, wi, accumulate=m > 0)
            qs.qs_synchronize(dm.handle)
            sv.close()
        assert maxdiff(dm.get_amps(), want) <= ATOL[arith], arith
        dms[arith] = dm
    u = wl.haar_unitary(4, rng)
    kraus = wl.haar_kraus(1, 2, rng)
    ops = [
        (lambda h: qs.qs_apply_depolarising(h, 3, 0.2), lambda b: orc.densmatr_apply_depolarising(b, 3, 0.2)),
        (lambda h: qs.qs_apply_dephasing(h, 12, 0.3), lambda b: orc.densmatr_apply_dephasing(b, 12, 0.3)),
        (lambda h: qs.qs_apply_damping(h, 0, 0.25), lambda b: orc.densmatr_apply_damping(b, 0, 0.25)),
        (lambda h: qs.qs_apply_pauli_channel(h, 7, 0.1, 0.05, 0.15),
         lambda b: orc.densmatr_apply_pauli_channel(b, 7, 0.1, 0.05, 0.15)),
        (lambda h: qs.qs_apply_kraus(h, [6], kraus), lambda b: orc.densmatr_apply_kraus(b, [6], kraus)),
        (lambda h: qs.qs_apply_ctrl_multi_target(h, [5], [9, 2], u),
         lambda b: orc.densmatr_apply_ctrl_multi_target(b, [5], [9, 2], u)),
    ]
    for k, (gpu_fn, orc_fn) in enumerate(ops):
        want = orc_fn(want)
        for arith, dm in dms.items():
            gpu_fn(dm.handle)
            err = maxdiff(dm.get_amps(), want)
            assert err <= ATOL[arith], (k, arith, err)
    want_red = orc.partial_trace(want, [4])
    want_tr = orc.calc_trace(want)
    for arith, dm in dms.items():
        red = dm.partial_trace([4])
        assert maxdiff(red.get_amps(), want_red) <= ATOL[arith], arith
        assert abs(qs.qs_calc_norm_or_trace(dm.handle) - want_tr) < STOL[arith], arith
        red.close()
        dm.close()


def _gather(psi_t, idx, stream):
    import torch
    with torch.cuda.stream(stream):
        out = psi_t[torch.from_numpy(np.asarray(idx, dtype=np.int64)).to(psi_t.device)].cpu().numpy()
    return out.astype(np.complex128)


@pytest.mark.parametrize("arith", ["fx", "df"])
def test_densmatr_14_qubits_two_qubit_ops_sampled(qs, arith):
    """Two-qubit depolarising and dephasing (2^24 groups of 16), a
    two-qubit Kraus map (its 16 x 16 superoperator on four targets) and a
    one-qubit Pauli channel on a 28-qubit Choi vector (4 GiB) of random
    amplitudes, each checked at 256 random outputs and the first and last
    indices against the oracle's single-output forms."""
    import torch
    nq = 14
    dim2 = 1 << (2 * nq)
    device = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=device)
    g = torch.Generator(device=device)
    g.manual_seed(2311015114)
    with torch.cuda.stream(stream):
        beta = torch.randn(dim2, dtype=torch.complex128, device=device, generator=g) * 2.0 ** -14
    stream.synchronize()
    dm = qs.State(nq, density=True, prec=qs.QS_C128, stream=stream, storage=beta)
    qs.qs_set_arithmetic(dm.handle, arith_code(qs, arith))
    rng = np.random.default_rng(1414)
    kraus = wl.haar_kraus(2, 4, rng)
    sup = orc.superoperator(kraus)
    cases = [
        ("depolarising2", (3, 11, 0.4)),
        ("dephasing2", (13, 0, 0.35)),
        ("kraus2", ([9, 1],)),
        ("pauli", (12, 0.1, 0.2, 0.05)),
    ]
    for name, args in cases:
        out_idx = np.concatenate([[0, dim2 - 1], rng.choice(dim2, 256, replace=False)]).astype(np.int64)
        if name == "depolarising2":
            t1, t2, p = args
            f1, f2 = (1 << t1) | (1 << (t1 + nq)), (1 << t2) | (1 << (t2 + nq))
            need = np.unique(np.concatenate([out_idx, out_idx ^ f1, out_idx ^ f2, out_idx ^ f1 ^ f2]))
        elif name == "pauli":
            t = args[0]
            need = np.unique(np.concatenate([out_idx, out_idx ^ ((1 << t) | (1 << (t + nq)))]))
        elif name == "kraus2":
            t4 = args[0] + [q + nq for q in args[0]]
            m4 = orc.get_bit_mask(t4)
            need = np.unique(np.array([orc.set_bits(int(i) & ~m4, t4, l) for i in out_idx for l in range(16)],
                                      dtype=np.int64))
        else:
            need = out_idx
        old = _gather(beta, need, stream)
        lookup = dict(zip(need.tolist(), old))
        get = lambda ix: np.array([lookup[int(i)] for i in np.atleast_1d(ix)], dtype=np.complex128)
        if name == "depolarising2":
            qs.qs_apply_two_qubit_depolarising(dm.handle, *args)
            want = orc.sample_densmatr_two_qubit_depolarising(get, nq, *args, out_idx)
        elif name == "dephasing2":
            qs.qs_apply_two_qubit_dephasing(dm.handle, *args)
            want = orc.sample_densmatr_two_qubit_dephasing(get, nq, *args, out_idx)
        elif name == "kraus2":
            qs.qs_apply_kraus(dm.handle, args[0], kraus)
            want = orc.sample_ctrl_multi_target(get, [], t4, sup, out_idx)
        else:
            qs.qs_apply_pauli_channel(dm.handle, *args)
            want = orc.sample_densmatr_pauli_channel(get, nq, *args, out_idx)
        qs.qs_synchronize(dm.handle)
        new = _gather(beta, out_idx, stream)
        scale = float(np.max(np.abs(old)))
        # the per-operation bounds of the small tests, relative to the
        # amplitudes' size here (about 2^-14)
        rel = 2.0 ** -47 if arith == "fx" else 2.0 ** -40
        err = maxdiff(new, want)
        assert err <= rel * scale, (name, arith, err, scale)
    dm.close()
    del beta
    torch.cuda.empty_cache()


def test_densmatr_expectation_320_terms(qs):
    """Tr(H rho) of a 10-qubit density matrix with 320 random Pauli terms:
    320 2^10 work items, more than the 1216 x 256 threads of the reduction."""
    rng = np.random.default_rng(1010)
    nq = 10
    states, w = wl.random_mixed_state_vectors(nq, 3, rng)
    beta = sum(wi * orc.densmatr_from_pure(s) for wi, s in zip(w, states))
    paulis, coeffs = wl.random_pauli_sum(nq, 320, rng)
    want = orc.expec_pauli_sum_densmatr(beta, paulis, coeffs)
    for arith in ("fx", "df"):
        dm = qs.State(nq, density=True, prec=qs.QS_C128)
        qs.qs_set_arithmetic(dm.handle, arith_code(qs, arith))
        dm.set_amps(beta)
        got = qs.qs_expec_pauli_sum(dm.handle, paulis, coeffs)
        assert abs(got - want) < STOL[arith] * np.abs(coeffs).sum(), (arith, got, want)
        dm.close()
