"""Batched-engine measurement: 4096 statevectors of 10-20 qubits (uniform
qubit counts), each with its own seeded circuit of 100-400 unitary
operations (one-qubit Haar unitaries, 1-2-target Haar unitaries with 0-3
controls, Pauli gadgets of weight 1-6), run as one recorded persistent launch
(qs_batch_*), against launching each circuit's operations separately through
the per-operation API on the same states.

    python -m paper_2311_01512_gb300.batch_bench [--prec 0|1] [--states S] [--reps R]

Prints one JSON line: the replay time (CUDA events, mean of R replays after
one untimed replay), gates/s, the chosen launch shape, and the per-circuit
baseline time."""

import argparse
import json
import sys
import time

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--prec", type=int, default=0, help="0 complex64, 1 complex128")
    ap.add_argument("--states", type=int, default=4096)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--no-baseline", action="store_true")
    args = ap.parse_args(argv)

    import torch
    from paper_2311_01512_gb300 import qs, workloads as wl

    rng = wl.rng_for("batch-bench")
    S = args.states
    sizes = [int(x) for x in rng.integers(10, 21, size=S)]
    nops = [int(x) for x in rng.integers(100, 401, size=S)]
    stream = torch.cuda.Stream()
    batch = qs.Batch(sizes, prec=args.prec, stream=stream)
    circs = []
    t0 = time.time()
    for s in range(S):
        ops = wl.unitary_circuit(sizes[s], nops[s], rng)
        circs.append(ops)
        for op in ops:
            batch.add(s, op)
    build_s = time.time() - t0
    t0 = time.time()
    batch.compile(autotune=True)
    compile_s = time.time() - t0
    info = batch.info()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    batch.run()
    stream.synchronize()
    e0.record(stream)
    for _ in range(args.reps):
        batch.run()
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / args.reps
    gates = sum(nops)
    out = {"states": S, "prec": "complex128" if args.prec == 1 else "complex64", "gates": gates,
           "replay_ms": ms, "gates_per_s": gates / ms * 1e3,
           "amplitude_updates_per_s": sum((1 << n) * k for n, k in zip(sizes, nops)) / ms * 1e3,
           "launch": info, "host_build_s": build_s, "compile_autotune_s": compile_s}
    if not args.no_baseline:
        hs = [qs.qs_create_statevector(sizes[s], args.prec, batch.view(s).data_ptr(), stream.cuda_stream)
              for s in range(S)]
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
    print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
