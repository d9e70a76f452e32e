"""Fixed sequence of hot-path kernel launches for profiling (ncu) at a chosen
size, in the default complex128 arithmetic (block fixed point): one-target
gate, 3-qubit diagonal, weight-6 Pauli gadget, a Z-only (phase) gadget, dense
gates on 2 targets (CUDA cores, block fixed point) and on 3, 4 and 5 targets
(bf16 tensor cores, eight integer slices), and a 5-target dense gate on a
complex64 state (tf32 tensor cores), each repeated.

    python -m paper_2311_01512_gb300.profile_ops --qubits 28 --reps 3

With --traffic-csv it instead turns ncu CSVs of dram__bytes_read.sum and
dram__bytes_write.sum (one capture per kernel, each over one repetition of
that sequence) into DRAM bytes per launch, scaled to a full pass over
--scale-to qubits (traffic grows with the amplitudes processed), keyed by the
bench's kernel families and stamped with the kernel sources' digest:

    python -m paper_2311_01512_gb300.profile_ops --qubits 28 --traffic-csv t_gate1.csv t_diag.csv ... \
        --scale-to 30 --out profiles/dram_traffic.json

With --dense-times it instead times complex128 dense gates (block fixed
point: the two-target CUDA-core kernel, eight-slice tensor-core kernels for
three to five targets) on a state of --qubits qubits at
three placements per target count (lowest qubits, spread, highest qubits)
and one controlled case, each the median of --reps CUDA-event timings after
one untimed launch, and prints ms and GB/s of amplitudes read and written:

    python -m paper_2311_01512_gb300.profile_ops --qubits 30 --reps 5 --dense-times

With --expec-times it instead times the statevector Pauli-sum expectation
(qs_expec_pauli_sum, wall clock around the synchronous call, median of
--reps after one untimed call) on a seeded complex128 state of --qubits
qubits with 8 and 100 random terms, in block fixed point (native FP64
reduction) and in double-float:

    python -m paper_2311_01512_gb300.profile_ops --qubits 28 --reps 5 --expec-times

With --all it instead launches every kernel family of the library once, on
a statevector of --qubits qubits in both precisions and a density matrix of
--qubits / 2 qubits (its Choi vector as large): the streaming gates, the
dense gates on 2-6 targets, SWAP, the channels, the superoperator and
Kraus map, the partial trace, the expectation kernels, norm and trace, the
fused-block composition.  It is the sequence for a per-kernel table of DRAM
bytes and times.
"""

import argparse
import csv
import json

import numpy as np

# launch order of one repetition -> the bench's kernel family names
_FAMILIES = {"k_gate1_fx": ["k_gate1"], "k_diag_fx": ["k_diag"], "k_gadget_fx": ["k_gadget"],
             "k_phase_fx": ["k_phase"], "k_gate2_fx": ["k_dense<2>"], "k_dense_ozaki_ws<3": ["k_dense<3>"],
             "k_dense_ozaki_ws<4": ["k_dense<4>"], "k_dense_ozaki<5": ["k_dense<5>"], "k_dense_tc<5": ["c64 k_dense<5>"]}


def summarize_traffic(paths, qubits, scale_to, out):
    from . import build
    launches = {}
    for n, path in enumerate(paths):
        rows = list(csv.reader(open(path)))
        hi = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
        hdr = rows[hi]
        ki, mi, vi, ii = (hdr.index("Kernel Name"), hdr.index("Metric Name"), hdr.index("Metric Value"),
                          hdr.index("ID"))
        for r in rows[hi + 1:]:
            if len(r) <= vi:
                continue
            d = launches.setdefault((n, r[ii]), {"name": r[ki].split("(")[0].replace("void ", "").replace("qsk::", "")})
            d[r[mi]] = float(r[vi].replace(",", ""))
    scale = 2.0 ** (scale_to - qubits)
    fam, pending = {}, {k: list(v) for k, v in _FAMILIES.items()}
    for d in launches.values():
        for prefix, names in pending.items():
            if d["name"].startswith(prefix) and names:
                b = d.get("dram__bytes_read.sum", 0.0) + d.get("dram__bytes_write.sum", 0.0)
                fam[names.pop(0)] = b * scale
                break
    rec = {"sources_sha256": build.sources_digest(), "measured_qubits": qubits, "scaled_to_qubits": scale_to,
           "unit": "bytes per full-pass launch (dram__bytes_read.sum + dram__bytes_write.sum)",
           "families": fam}
    with open(out, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec, indent=1))


def dense_times(nq, reps):
    import torch
    from . import qs
    from . import workloads as wl
    st = qs.State(nq, density=False, prec=qs.QS_C128)
    st.tensor.real.normal_()
    st.tensor.imag.normal_()
    st.tensor /= torch.linalg.vector_norm(st.tensor)
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    spread = [0, 4, 9, 17, 25]
    cases = {n: [list(range(n)), spread[:n] if n > 2 else [3, 9], list(range(nq - n, nq))] for n in (2, 3, 4, 5)}

    def timed(ctrls, targs, u):
        ts = []
        for r in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st.stream)
            qs.qs_apply_ctrl_multi_target(st.handle, ctrls, targs, u)
            e1.record(st.stream)
            e1.synchronize()
            if r:
                ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    nbytes = 2 * 16 * (1 << nq)
    for n, placements in cases.items():
        u = wl.haar_unitary(1 << n, rng)
        for targs in placements:
            ms = timed([], targs, u)
            print("%d targets %-18s %8.3f ms %8.1f GB/s" % (n, targs, ms, nbytes / ms / 1e6))
        c = [q for q in range(nq) if q not in placements[1]][-1]
        ms = timed([c], placements[1], u)
        print("%d targets %-18s %8.3f ms %8.1f GB/s (control %d)" % (n, placements[1], ms, nbytes / 2 / ms / 1e6, c))
    print("norm", qs.qs_calc_norm_or_trace(st.handle).real)
    st.close()


def expec_times(nq, reps):
    import time
    import torch
    from . import qs
    from . import workloads as wl
    stream = torch.cuda.Stream()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    with torch.cuda.stream(stream):
        psi = torch.randn(1 << nq, dtype=torch.complex128, device="cuda", generator=gen)
        psi /= torch.linalg.vector_norm(psi)
    stream.synchronize()
    st = qs.State(nq, prec=qs.QS_C128, stream=stream, storage=psi)
    rng = np.random.default_rng(1)
    out = {}
    for arith, code in (("fx", qs.QS_ARITH_FX), ("df", qs.QS_ARITH_DF)):
        qs.qs_set_arithmetic(st.handle, code)
        for nterms in (8, 100):
            paulis, coeffs = wl.random_pauli_sum(nq, nterms, rng)
            qs.qs_expec_pauli_sum(st.handle, paulis, coeffs)
            ts = []
            for _ in range(reps):
                t0 = time.perf_counter()
                v = qs.qs_expec_pauli_sum(st.handle, paulis, coeffs)
                ts.append(time.perf_counter() - t0)
            out["%s_%d_terms" % (arith, nterms)] = {"ms_median": round(1e3 * float(np.median(ts)), 3),
                                                     "value": float(v.real)}
    print(json.dumps(out))
    st.close()


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--qubits", type=int, default=28)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--traffic-csv", nargs="+")
    ap.add_argument("--scale-to", type=int, default=30)
    ap.add_argument("--out", default="profiles/dram_traffic.json")
    ap.add_argument("--all", action="store_true")
    ap.add_argument("--dense-times", action="store_true")
    ap.add_argument("--expec-times", action="store_true")
    args = ap.parse_args(argv)
    if args.expec_times:
        expec_times(args.qubits, args.reps)
        return
    if args.dense_times:
        dense_times(args.qubits, args.reps)
        return
    if args.traffic_csv:
        summarize_traffic(args.traffic_csv, args.qubits, args.scale_to, args.out)
        return
    if args.all:
        every_kernel(args.qubits)
        return
    import torch
    from . import qs
    from . import workloads as wl
    nq = args.qubits
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        psi = torch.randn(1 << nq, dtype=torch.complex128, device="cuda")
        psi /= torch.linalg.vector_norm(psi)
        p64 = psi.to(torch.complex64)
    stream.synchronize()
    s128 = qs.State(nq, prec=qs.QS_C128, stream=stream, storage=psi)
    s64 = qs.State(nq, prec=qs.QS_C64, stream=stream, storage=p64)
    rng = np.random.default_rng(3)
    u = wl.haar_unitary(2, rng)
    mats = {n: wl.haar_unitary(1 << n, rng) for n in (2, 3, 4, 5)}
    targets = {2: [5, 19], 3: [2, 13, 21], 4: [2, 9, 13, 21], 5: [0, 4, 9, 17, nq - 2]}
    diag = np.exp(1j * rng.uniform(0, 2 * np.pi, 8))
    for _ in range(args.reps):
        qs.qs_apply_ctrl_multi_target(s128.handle, [], [17], u)
        qs.qs_apply_diagonal(s128.handle, [1, 7, 20], diag)
        qs.qs_apply_pauli_gadget(s128.handle, [0, 3, 8, 15, 22, nq - 1], [1, 2, 3, 1, 2, 3], 0.4)
        qs.qs_apply_pauli_gadget(s128.handle, [0, 4, 9, 17], [3, 3, 3, 3], 0.4)
        for n in (2, 3, 4, 5):
            qs.qs_apply_ctrl_multi_target(s128.handle, [], targets[n], mats[n])
        qs.qs_apply_ctrl_multi_target(s64.handle, [], targets[5], mats[5])
    stream.synchronize()
    print("norms", qs.qs_calc_norm_or_trace(s128.handle).real, qs.qs_calc_norm_or_trace(s64.handle).real)
    s128.close()
    s64.close()


def every_kernel(nq):
    import torch
    from . import qs
    from . import workloads as wl
    stream = torch.cuda.Stream()
    rng = np.random.default_rng(4)
    with torch.cuda.stream(stream):
        psi = torch.randn(1 << nq, dtype=torch.complex128, device="cuda")
        psi /= torch.linalg.vector_norm(psi)
    stream.synchronize()
    u = wl.haar_unitary(2, rng)
    mats = {n: wl.haar_unitary(1 << n, rng) for n in range(2, 7)}
    targets = {2: [5, 19], 3: [2, 13, 21], 4: [2, 9, 13, 21], 5: [0, 4, 9, 17, nq - 2], 6: [1, 4, 9, 12, 17, nq - 3]}
    diag = np.exp(1j * rng.uniform(0, 2 * np.pi, 8))
    paulis, coeffs = wl.random_pauli_sum(nq, 8, rng)
    zs = np.where(rng.random((16, nq)) < 0.4, 3, 0).astype(np.int32)
    for prec in (qs.QS_C128, qs.QS_C64):
        with torch.cuda.stream(stream):
            t = psi if prec == qs.QS_C128 else psi.to(torch.complex64)
        stream.synchronize()
        st = qs.State(nq, prec=prec, stream=stream, storage=t)
        h = st.handle
        qs.qs_apply_ctrl_multi_target(h, [], [17], u)                       # one-target gate
        qs.qs_apply_diagonal(h, [1, 7, 20], diag)                            # diagonal
        qs.qs_apply_pauli_gadget(h, [0, 3, 8, 15, 22, nq - 1], [1, 2, 3, 1, 2, 3], 0.4)   # gadget
        qs.qs_apply_pauli_gadget(h, [0, 4, 9, 17], [3, 3, 3, 3], 0.4)        # phase gadget
        for n in range(2, 7 if prec == qs.QS_C64 else 6):
            qs.qs_apply_ctrl_multi_target(h, [], targets[n], mats[n])        # dense gates (c128 2: CUDA cores)
        qs.qs_apply_swap(h, 3, 17)
        qs.qs_expec_pauli_sum(h, paulis, coeffs)                             # off-diagonal terms
        qs.qs_expec_pauli_sum(h, zs, rng.standard_normal(16))                # Walsh-Hadamard diagonal terms
        qs.qs_calc_norm_or_trace(h)
        st.close()
        del t
    # fused blocks: FP64 composition, then the blocks
    circ = qs.Circuit(nq, wl.unitary_circuit(nq, 12, rng))
    circ.plan(qs.QS_PLAN_GREEDY, 4)
    st = qs.State(nq, prec=qs.QS_C128, stream=stream, storage=psi)
    circ.apply(st.handle)
    qs.qs_synchronize(st.handle)
    st.close()
    circ.close()
    del psi
    torch.cuda.empty_cache()
    # density matrix of nq / 2 qubits
    nd = nq // 2
    rho = qs.State(nd, density=True, prec=qs.QS_C128, stream=stream)
    sv = qs.State(nd, prec=qs.QS_C128, stream=stream)
    sv.set_amps(wl.random_statevector(nd, rng))
    qs.qs_init_pure_densmatr(rho.handle, sv.handle, 1.0, 0)
    h = rho.handle
    qs.qs_apply_dephasing(h, 1, 0.05)
    qs.qs_apply_two_qubit_dephasing(h, 1, 5, 0.05)
    qs.qs_apply_depolarising(h, 2, 0.05)
    qs.qs_apply_two_qubit_depolarising(h, 2, 6, 0.05)
    qs.qs_apply_damping(h, 3, 0.05)
    qs.qs_apply_pauli_channel(h, 4, 0.02, 0.03, 0.01)
    qs.qs_apply_kraus(h, [0, 7], wl.haar_kraus(2, 4, rng))                   # superoperator + 4-target pass
    qs.qs_apply_ctrl_multi_target(h, [], [1, 6], mats[2])                    # one superoperator pass
    pd, cd = wl.random_pauli_sum(nd, 20, rng)
    qs.qs_expec_pauli_sum(h, pd, cd)
    red = rho.partial_trace([1, 4, 7])
    qs.qs_calc_norm_or_trace(h)
    red.close()
    rho.close()
    sv.close()
    print("every kernel launched")


if __name__ == "__main__":
    main()
