"""Density-matrix workloads end to end on one GPU (complex128, CUDA events):

* 6 qubits (a 12-qubit Choi vector, 64 KiB): a rank-4 mixture, 300 operations
  of workloads.small_densmatr_circuit (Haar unitaries, gadgets, depolarising,
  damping, 2-qubit 4-Kraus channels), a partial trace over 2 qubits and a
  20-term Pauli sum.  The state stays in L2, so the figure is microseconds per
  operation (launch-bound).
* 15 qubits (a 30-qubit Choi vector, 16 GiB): a rank-8 mixture, 400
  operations of workloads.large_densmatr_circuit (Haar unitaries on 1-3
  targets with 0-3 controls, 1q/2q depolarising and dephasing, damping,
  2-qubit 4-Kraus channels), a partial trace of 5 qubits and a 100-term Pauli
  sum.  Reported per operation kind: launches, time, the algorithmic bytes
  (each amplitude a pass touches read and written once) and their rate.

    python -m paper_2311_01512_gb300.dm_bench [--small-reps R] [--large-reps R] [--no-large]

Prints one JSON line per workload."""

import argparse
import json
import sys

import numpy as np


def _events(torch, n):
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def mixture(qs, wl, nq, rank, rng, stream):
    rho = qs.State(nq, density=True, prec=qs.QS_C128, stream=stream)
    w = wl.random_mixture_weights(rank, rng)
    for m in range(rank):
        sv = qs.State(nq, density=False, prec=qs.QS_C128, stream=stream)
        sv.set_amps(wl.random_statevector(nq, rng))
        qs.qs_init_pure_densmatr(rho.handle, sv.handle, float(w[m]), accumulate=m > 0)
        qs.qs_synchronize(rho.handle)
        sv.close()
    return rho


def op_bytes(op, nq):
    """Algorithmic bytes of one operation on a Choi vector of 2 nq qubits."""
    full = 32 * (1 << (2 * nq))
    kind = op["op"]
    if kind == "unitary":
        s = len(op["ctrls"])
        if s == 0 and len(op["targs"]) <= 2:
            return full                     # one pass of conj(U) (x) U on 2 or 4 targets
        return 2 * full >> s                # U on t, then U* on t + N
    if kind == "gadget":
        return 2 * full
    if kind == "dephasing":
        return full // 2                    # scales the half whose two bits differ
    if kind == "dephasing2":
        return full * 3 // 4
    return full


def small(qs, wl, torch, reps):
    nq = 6
    rng = wl.rng_for("dm6-bench")
    stream = torch.cuda.Stream()
    rho = mixture(qs, wl, nq, 4, rng, stream)
    ops = wl.small_densmatr_circuit(nq, 300, rng)
    paulis, coeffs = wl.random_pauli_sum(nq, 20, rng)
    e0, e1 = _events(torch, 2)

    def run():
        for op in ops:
            qs.apply_op(rho.handle, op)
        red = rho.partial_trace([1, 4])
        val = qs.qs_expec_pauli_sum(rho.handle, paulis, coeffs)
        red.close()
        return val

    run()
    stream.synchronize()
    e0.record(stream)
    for _ in range(reps):
        val = run()
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / reps
    # the same 300 operations recorded once and replayed as one graph launch
    qs.qs_record_begin(rho.handle)
    for op in ops:
        qs.apply_op(rho.handle, op)
    prog = qs.qs_record_end(rho.handle)
    qs.qs_program_run(prog)
    stream.synchronize()
    e0.record(stream)
    for _ in range(reps):
        qs.qs_program_run(prog)
    e1.record(stream)
    e1.synchronize()
    prog_ms = e0.elapsed_time(e1) / reps
    qs.qs_program_destroy(prog)
    # the same 300 operations as a batch of one state: one persistent launch
    # that keeps the Choi vector in shared memory for the whole circuit
    batch = qs.Batch([nq], prec=qs.QS_C128, stream=stream, density=[True])
    for op in ops:
        batch.add(0, op)
    batch.compile(autotune=True)
    batch.view(0).copy_(rho.tensor)
    batch.run()
    stream.synchronize()
    e0.record(stream)
    for _ in range(reps):
        batch.run()
    e1.record(stream)
    e1.synchronize()
    batch_ms = e0.elapsed_time(e1) / reps
    batch.close()
    return {"workload": "6-qubit density matrix (12-qubit Choi vector), 300 ops + partial trace + 20-term sum",
            "ms_per_run": ms, "us_per_op": ms * 1e3 / (len(ops) + 2), "reps": reps,
            "recorded_ms_per_300_ops": prog_ms, "recorded_us_per_op": prog_ms * 1e3 / len(ops),
            "batched_ms_per_300_ops": batch_ms, "batched_us_per_op": batch_ms * 1e3 / len(ops),
            "trace": qs.qs_calc_norm_or_trace(rho.handle).real, "expectation": val.real}


def large(qs, wl, torch, peak_gbs, reps=1):
    """The 400-operation circuit `reps` times on the evolving state (the
    channels keep the trace, the unitaries the spectrum); times per kind from
    the last run, the circuit time as the median over runs."""
    nq = 15
    rng = wl.rng_for("dm15-bench")
    stream = torch.cuda.Stream()
    rho = mixture(qs, wl, nq, 8, rng, stream)
    ops = wl.large_densmatr_circuit(nq, 400, rng)
    ev = _events(torch, len(ops) + 1)
    totals = []
    for _ in range(reps):
        ev[0].record(stream)
        for k, op in enumerate(ops):
            qs.apply_op(rho.handle, op)
            ev[k + 1].record(stream)
        ev[-1].synchronize()
        totals.append(ev[0].elapsed_time(ev[-1]))
    fam = {}
    for k, op in enumerate(ops):
        kind = op["op"]
        if kind == "unitary":
            kind = "unitary %dq%s" % (len(op["targs"]), " controlled" if op["ctrls"] else "")
        ms = ev[k].elapsed_time(ev[k + 1])
        f = fam.setdefault(kind, {"launches": 0, "ms": 0.0, "bytes": 0})
        f["launches"] += 1
        f["ms"] += ms
        f["bytes"] += op_bytes(op, nq)
    total_ms = float(np.median(totals))
    total_bytes = sum(f["bytes"] for f in fam.values())
    for f in fam.values():
        f["gbs"] = f["bytes"] / f["ms"] / 1e6
        f["frac_of_peak"] = f["gbs"] / peak_gbs if peak_gbs else None
    e0, e1 = _events(torch, 2)
    for _ in range(2):                      # the second call is timed (the first allocates)
        e0.record(stream)
        red = rho.partial_trace([1, 4, 7, 10, 13])
        e1.record(stream)
        e1.synchronize()
        pt_ms = e0.elapsed_time(e1)
        if _ == 0:
            red.close()
    paulis, coeffs = wl.random_pauli_sum(nq, 100, rng)
    for _ in range(2):
        e0.record(stream)
        val = qs.qs_expec_pauli_sum(rho.handle, paulis, coeffs)
        e1.record(stream)
        e1.synchronize()
        ex_ms = e0.elapsed_time(e1)
    out = {"workload": "15-qubit density matrix (30-qubit Choi vector, 16 GiB), 400 ops",
           "arithmetic": "complex128, the default block fixed point (two-target passes on the CUDA cores, "
                         "3-5-target passes as eight slices on the tensor cores)",
           "runs": reps, "ms_total": total_ms, "ms_runs": totals, "gb_total": total_bytes / 1e9,
           "gbs": total_bytes / total_ms / 1e6,
           "frac_of_peak": (total_bytes / total_ms / 1e6) / peak_gbs if peak_gbs else None,
           "by_kind": fam, "partial_trace_5q_ms": pt_ms, "expectation_100_terms_ms": ex_ms,
           "trace": qs.qs_calc_norm_or_trace(rho.handle).real, "reduced_trace": qs.qs_calc_norm_or_trace(red.handle).real,
           "expectation": val.real}
    red.close()
    rho.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--small-reps", type=int, default=20)
    ap.add_argument("--no-large", action="store_true")
    ap.add_argument("--large-reps", type=int, default=3)
    args = ap.parse_args(argv)
    import os
    import torch
    from paper_2311_01512_gb300 import qs, workloads as wl
    peak = None
    pk = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        with open(pk) as f:
            peak = json.load(f).get("hbm_gbs")
    print(json.dumps(small(qs, wl, torch, args.small_reps)), flush=True)
    if not args.no_large:
        print(json.dumps(large(qs, wl, torch, peak, args.large_reps)), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
