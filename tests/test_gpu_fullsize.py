"""Full-size parity in the launch configuration bench.py times: the 30-qubit
complex128 state (16 GiB) and the first operations of the bench's 500-op
circuit, covering every kernel the circuit uses.  For each operation, outputs
at sampled indices are compared with the oracle evaluated one amplitude at a
time from the gathered old amplitudes; the norm is checked after all of them
(unitary circuit: preserved at any size)."""

import numpy as np
import pytest

from oracle import qsim_oracle as orc

pytestmark = pytest.mark.gpu

NQ = 30
SAMPLES = 192


def _partners(op, out_idx):
    """Old-amplitude indices the sampled outputs of op depend on."""
    idx = [int(i) for i in out_idx]
    if op["op"] == "unitary":
        n = len(op["targs"])
        tmask = orc.get_bit_mask(op["targs"])
        return sorted({orc.set_bits(i & ~tmask, op["targs"], l) for i in idx for l in range(1 << n)} | set(idx))
    if op["op"] == "gadget":
        xy, _, _ = orc._pauli_masks(op["targs"], op["paulis"])
        return sorted(set(idx) | {i ^ xy for i in idx})
    return sorted(set(idx))


def test_bench_circuit_sampled_parity_at_30_qubits():
    import torch
    import bench
    from paper_2311_01512_gb300 import qs
    device = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=device)
    with torch.cuda.stream(stream):
        psi = bench.device_random_state(NQ, device)
    stream.synchronize()
    st = qs.State(NQ, prec=qs.QS_C128, stream=stream, storage=psi)
    ops = bench.make_ops(NQ)
    # the first operation of every kernel family in the circuit, in order
    chosen, seen = [], set()
    for k, op in enumerate(ops):
        fam = bench.op_family(op)
        if fam not in seen:
            seen.add(fam)
            chosen.append(k)
    rng = np.random.default_rng(30)
    for k in range(max(chosen) + 1):
        op = ops[k]
        if k in chosen:
            out_idx = rng.choice(1 << NQ, SAMPLES, replace=False)
            need = np.array(_partners(op, out_idx), dtype=np.int64)
            with torch.cuda.stream(stream):
                old = psi[torch.from_numpy(need).to(device)].cpu().numpy()
            lookup = dict(zip(need.tolist(), old))
            get = lambda ix: np.array([lookup[int(i)] for i in ix], dtype=np.complex128)
        qs.apply_op(st.handle, op)
        if k in chosen:
            qs.qs_synchronize(st.handle)
            with torch.cuda.stream(stream):
                new = psi[torch.from_numpy(out_idx).to(device)].cpu().numpy()
            if op["op"] == "unitary":
                want = orc.sample_ctrl_multi_target(get, op["ctrls"], op["targs"], op["mat"], out_idx)
            elif op["op"] == "diagonal":
                want = orc.sample_diagonal(get, op["targs"], op["diag"], out_idx)
            else:
                want = orc.sample_pauli_gadget(get, op["targs"], op["paulis"], op["theta"], out_idx)
            err = float(np.max(np.abs(new - want)))
            # block fixed point (the default arithmetic): one output is within
            # 2^-53 |y| + 2^-55 max|x| max|m| (K <= 4 terms), and a dense gate
            # of n <= 5 targets within (2^(n+1) + 1) 2^-54 <= 2^-48 of the
            # largest amplitude it combines (unitary rows: entries <= 1); the
            # oracle's own FP64 evaluation adds a few 2^-53
            assert err <= 2.0 ** -47 * float(np.max(np.abs(old))), (k, bench.op_family(op), err)
    assert abs(qs.qs_calc_norm_or_trace(st.handle).real - 1.0) < 1e-13
    assert len(seen) >= 5
    st.close()


def test_large_density_matrix_properties_at_15_qubits():
    """15-qubit density matrix held as a 30-qubit Choi vector (16 GiB): rank-8
    mixture, 40 operations of the large density workload (Haar unitaries with
    controls, 1q/2q depolarising and dephasing, damping, 2-qubit Kraus
    channels), then a partial trace of 5 qubits and a 100-term Pauli sum.
    Properties that hold at any size: trace preserved by every channel,
    rho_kl = conj(rho_lk) at sampled pairs, the reduced state keeps the
    trace, and Tr(H rho) is real."""
    import torch
    from paper_2311_01512_gb300 import qs
    from paper_2311_01512_gb300 import workloads as wl
    nq = 15
    rng = wl.rng_for("dm15-fullsize")
    stream = torch.cuda.Stream()
    rho = qs.State(nq, density=True, prec=qs.QS_C128, stream=stream)
    w = wl.random_mixture_weights(8, rng)
    for m in range(8):
        sv = qs.State(nq, density=False, prec=qs.QS_C128, stream=stream)
        sv.set_amps(wl.random_statevector(nq, rng))
        qs.qs_init_pure_densmatr(rho.handle, sv.handle, float(w[m]), accumulate=m > 0)
        qs.qs_synchronize(rho.handle)
        sv.close()
    assert abs(qs.qs_calc_norm_or_trace(rho.handle) - 1.0) < 1e-13
    for op in wl.large_densmatr_circuit(nq, 40, rng):
        qs.apply_op(rho.handle, op)
    tr = qs.qs_calc_norm_or_trace(rho.handle)
    assert abs(tr - 1.0) < 1e-12, tr
    dim = 1 << nq
    k = rng.integers(0, dim, 256)
    l = rng.integers(0, dim, 256)
    t = rho.tensor
    with torch.cuda.stream(stream):
        a = t[torch.from_numpy(k + l * dim).cuda()].cpu().numpy()
        b = t[torch.from_numpy(l + k * dim).cuda()].cpu().numpy()
    assert float(np.max(np.abs(a - np.conj(b)))) < 1e-15
    red = rho.partial_trace([int(x) for x in rng.choice(nq, 5, replace=False)])
    assert abs(qs.qs_calc_norm_or_trace(red.handle) - tr) < 1e-12
    paulis, coeffs = wl.random_pauli_sum(nq, 100, rng)
    e = qs.qs_expec_pauli_sum(rho.handle, paulis, coeffs)
    assert abs(e.imag) < 1e-12
    red.close()
    rho.close()


def test_indices_beyond_32_bits_complex64_33_qubits():
    """A 33-qubit complex64 state (64 GiB), so that amplitude indices pass
    2^32: one-target, dense (tensor-core) and 2-target gates, a diagonal, a
    gadget and a SWAP, each touching qubit 32, with outputs sampled at random
    indices and at 0, 2^32 - 1, 2^32, 2^32 + 1 and 2^33 - 1, against the
    oracle evaluated one amplitude at a time."""
    import torch
    from paper_2311_01512_gb300 import qs
    from paper_2311_01512_gb300 import workloads as wl
    nq = 33
    device = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=device)
    g = torch.Generator(device=device)
    g.manual_seed(2311015133)
    with torch.cuda.stream(stream):
        psi = torch.randn(1 << nq, dtype=torch.complex64, device=device, generator=g)
        psi /= torch.linalg.vector_norm(psi)
    stream.synchronize()
    st = qs.State(nq, prec=qs.QS_C64, stream=stream, storage=psi)
    rng = np.random.default_rng(33)
    ops = [
        {"op": "unitary", "ctrls": [], "targs": [32], "mat": wl.haar_unitary(2, rng)},
        {"op": "unitary", "ctrls": [31], "targs": [32, 5, 17], "mat": wl.haar_unitary(8, rng)},
        {"op": "unitary", "ctrls": [], "targs": [0, 32], "mat": wl.haar_unitary(4, rng)},
        {"op": "diagonal", "targs": [32, 0, 20], "diag": np.exp(1j * rng.uniform(0, 2 * np.pi, 8))},
        {"op": "gadget", "targs": [32, 1, 31], "paulis": [1, 2, 3], "theta": 0.7},
        {"op": "swap", "targs": [32, 3]},
    ]
    extremes = np.array([0, (1 << 32) - 1, 1 << 32, (1 << 32) + 1, (1 << nq) - 1], dtype=np.int64)
    for op in ops:
        out_idx = np.concatenate([extremes, rng.choice(1 << nq, 96, replace=False)])
        if op["op"] == "swap":
            t1, t2 = op["targs"]
            need = np.array(sorted(set(out_idx.tolist()) | {int(i) ^ ((1 << t1) | (1 << t2)) for i in out_idx}),
                            dtype=np.int64)
        else:
            need = np.array(_partners(op, out_idx), dtype=np.int64)
        with torch.cuda.stream(stream):
            old = psi[torch.from_numpy(need).to(device)].cpu().numpy().astype(np.complex128)
        lookup = dict(zip(need.tolist(), old))
        get = lambda ix: np.array([lookup[int(i)] for i in ix], dtype=np.complex128)
        qs.apply_op(st.handle, op)
        qs.qs_synchronize(st.handle)
        with torch.cuda.stream(stream):
            new = psi[torch.from_numpy(out_idx).to(device)].cpu().numpy().astype(np.complex128)
        if op["op"] == "unitary":
            want = orc.sample_ctrl_multi_target(get, op["ctrls"], op["targs"], op["mat"], out_idx)
        elif op["op"] == "diagonal":
            want = orc.sample_diagonal(get, op["targs"], op["diag"], out_idx)
        elif op["op"] == "gadget":
            want = orc.sample_pauli_gadget(get, op["targs"], op["paulis"], op["theta"], out_idx)
        else:
            want = orc.sample_swap(get, op["targs"][0], op["targs"][1], out_idx)
        err = float(np.max(np.abs(new - want)))
        # complex64 storage; 3xTF32 and FP32 arithmetic keep ~2^-21 of the amplitudes
        assert err <= 2.0 ** -19 * float(np.max(np.abs(old))), (op["op"], op["targs"], err)
    st.close()
    del psi
    torch.cuda.empty_cache()
