"""Batched-engine measurement: 4096 statevectors of 10-20 qubits (uniform
qubit counts), each with its own seeded circuit of 100-400 unitary
operations (one-qubit Haar unitaries, 1-2-target Haar unitaries with 0-3
controls, Pauli gadgets of weight 1-6), run as one recorded persistent launch
(qs_batch_*), against launching each circuit's operations separately through
the per-operation API on the same states.

    python -m paper_2311_01512_gb300.batch_bench [--prec 0|1] [--states S] [--reps R] [--fidelity-states F]

Prints one JSON line: the replay time (CUDA events, median of R replays after
one untimed replay), gates/s, the chosen launch shape, the per-circuit
baseline time and, with F > 0, 1 - fidelity of F sampled states against an
FP64-level reference (the per-operation path in block fixed point)."""

import argparse
import json
import sys
import time

import numpy as np


_WORKLOADS = {}


def workload(states, seed_tag):
    """Qubit counts, operation counts and seeded circuits of the batch (drawn
    once per process and shared by both precisions)."""
    key = (states, seed_tag)
    if key not in _WORKLOADS:
        from paper_2311_01512_gb300 import workloads as wl
        rng = wl.rng_for(seed_tag)
        sizes = [int(x) for x in rng.integers(10, 21, size=states)]
        nops = [int(x) for x in rng.integers(100, 401, size=states)]
        circs = [wl.unitary_circuit(sizes[s], nops[s], rng) for s in range(states)]
        _WORKLOADS[key] = (sizes, nops, circs)
    return _WORKLOADS[key]


def run(prec=0, states=4096, reps=3, baseline=True, fidelity_states=0, seed_tag="batch-bench"):
    """One measurement of the batched workload; returns a dict.

    The states start as normalised complex Gaussian vectors.  The replay time
    is the median of `reps` replays after one untimed replay.  The per-circuit
    baseline applies the same operations through the per-operation API on
    the same states (complex128 handles in the engine's double-float
    arithmetic).  With fidelity_states > 0, that many states (seeded choice)
    are reset to fresh random vectors, the batch is replayed once, and each
    is compared with its circuit applied through the per-operation API in
    complex128 block fixed point (FP64-level):
    1 - |<ref|gpu>|^2 / (|ref|^2 |gpu|^2) and max |delta amp|."""
    import torch
    from paper_2311_01512_gb300 import qs, workloads as wl

    t0 = time.time()
    sizes, nops, circs = workload(states, seed_tag)
    gen_s = time.time() - t0
    S = states
    stream = torch.cuda.Stream()
    batch = qs.Batch(sizes, prec=prec, stream=stream)
    t0 = time.time()
    for s in range(S):
        for op in circs[s]:
            batch.add(s, op)
    build_s = time.time() - t0
    t0 = time.time()
    batch.compile(autotune=True)
    compile_s = time.time() - t0
    info = batch.info()
    g = torch.Generator(device=batch.pool.device)
    g.manual_seed(2311015125)
    with torch.cuda.stream(stream):
        for s in range(S):
            v = batch.view(s)
            v.copy_(torch.randn(v.numel(), dtype=v.dtype, device=v.device, generator=g))
            v /= torch.linalg.vector_norm(v)
    stream.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    batch.run()
    stream.synchronize()
    times = []
    for _ in range(reps):
        e0.record(stream)
        batch.run()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = float(np.median(times))
    gates = sum(nops)
    out = {"states": S, "prec": "complex128" if prec == 1 else "complex64",
           "arithmetic": "double-float" if prec == 1 else "FP32 (float pairs)", "gates": gates,
           "qubits": "uniform over 10..20 per state (log-uniform amplitude counts)",
           "replay_ms": ms, "replay_ms_runs": times, "gates_per_s": gates / ms * 1e3,
           "amplitude_updates_per_s": sum((1 << n) * k for n, k in zip(sizes, nops)) / ms * 1e3,
           "launch": info, "host_generate_s": gen_s, "host_build_s": build_s, "compile_autotune_s": compile_s}
    if baseline:
        hs = [qs.qs_create_statevector(sizes[s], prec, batch.view(s).data_ptr(), stream.cuda_stream)
              for s in range(S)]
        if prec == 1:
            for h in hs:
                qs.qs_set_arithmetic(h, qs.QS_ARITH_DF)
        e0.record(stream)
        for s in range(S):
            for op in circs[s]:
                qs.apply_op(hs[s], op)
        e1.record(stream)
        e1.synchronize()
        base = e0.elapsed_time(e1)
        for h in hs:
            qs.qs_destroy(h)
        out["per_circuit_launches_ms"] = base
        out["speedup"] = base / ms
    if fidelity_states > 0:
        frng = np.random.default_rng(4096)
        pick = sorted(int(x) for x in frng.choice(S, min(fidelity_states, S), replace=False))
        refs = {}
        with torch.cuda.stream(stream):
            for s in pick:
                v = batch.view(s)
                v.copy_(torch.randn(v.numel(), dtype=v.dtype, device=v.device, generator=g))
                v /= torch.linalg.vector_norm(v)
                refs[s] = v.to(torch.complex128).clone()   # a copy even when v is already complex128
        stream.synchronize()
        batch.run()
        for s in pick:
            ref = qs.State(sizes[s], density=False, prec=qs.QS_C128, stream=stream, storage=refs[s])
            for op in circs[s]:
                qs.apply_op(ref.handle, op)
            ref.close()
        stream.synchronize()
        per = []
        for s in pick:
            got = batch.view(s).to(torch.complex128)
            want = refs[s]
            ov = torch.vdot(want, got)
            f = float(abs(ov) ** 2 / (torch.vdot(want, want).real * torch.vdot(got, got).real))
            per.append({"state": s, "qubits": sizes[s], "ops": nops[s], "one_minus_fidelity": 1.0 - f,
                        "max_abs_delta_amp": float((got - want).abs().max())})
        out["fidelity_sample"] = {
            "states": len(per), "choice": "seeded (numpy default_rng(4096)) among all states",
            "reference": ("the same circuit through the per-operation C ABI in complex128 block fixed point "
                          "(at least FP64; checked against the FP64 CPU oracle to 1e-14 per operation by the "
                          "parity tests)"),
            "max_one_minus_fidelity": max(p["one_minus_fidelity"] for p in per),
            "max_abs_delta_amp": max(p["max_abs_delta_amp"] for p in per), "per_state": per}
    batch.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--prec", type=int, default=0, help="0 complex64, 1 complex128")
    ap.add_argument("--states", type=int, default=4096)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--no-baseline", action="store_true")
    ap.add_argument("--fidelity-states", type=int, default=0)
    args = ap.parse_args(argv)
    out = run(args.prec, args.states, args.reps, not args.no_baseline, args.fidelity_states)
    print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
