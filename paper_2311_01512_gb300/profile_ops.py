"""Fixed sequence of hot-path kernel launches for profiling (ncu) at a chosen
size: one-target gate, 3-qubit diagonal, weight-6 Pauli gadget, dense gates
on 2 targets (complex128, double-float) and on 3, 4 and 5 targets (complex128,
bf16 tensor cores), and a 5-target dense gate on a complex64 state (tf32
tensor cores), each repeated.

    python -m paper_2311_01512_gb300.profile_ops --qubits 28 --reps 3
"""

import argparse

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--qubits", type=int, default=28)
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args(argv)
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
        for n in (2, 3, 4, 5):
            qs.qs_apply_ctrl_multi_target(s128.handle, [], targets[n], mats[n])
        qs.qs_apply_ctrl_multi_target(s64.handle, [], targets[5], mats[5])
    stream.synchronize()
    print("norms", qs.qs_calc_norm_or_trace(s128.handle).real, qs.qs_calc_norm_or_trace(s64.handle).real)
    s128.close()
    s64.close()


if __name__ == "__main__":
    main()
