"""Training data and training for the fusion cost model.

The simulator times its own kernel launches: random one-gate launches and
random fused-block launches (qs_apply_dense_block) on states of several sizes
and both precisions, each timed by CUDA events on the state's stream.  The
features of each launch come from the library's encoder (qs_costmodel_encode)
so that training and planning see identical rows; the target is log(ms).
Training runs on the GPU through qs_costmodel_train (the library's forward,
backward and Adam kernels).

    python -m paper_2311_01512_gb300.costmodel --samples 20000 --out costmodel_gb300.npz
"""

import argparse
import json
import math
import os
import time

import numpy as np

from . import workloads as wl

WEIGHTS_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "costmodel_gb300.npz")

# (kind name, probability): fused blocks dominate the planner's queries
KINDS = [("fused", 0.40), ("gate1", 0.15), ("dense", 0.15), ("diag", 0.10), ("gadget", 0.10), ("phase", 0.10)]


def _random_launch(qs, rng, nq):
    """One random launch: (callable on a handle, cost kind, width, qubit mask, controls, weight)."""
    r = rng.random()
    acc = 0.0
    for name, p in KINDS:
        acc += p
        if r <= acc:
            break
    if name == "fused":
        k = int(rng.integers(1, 7))
        targs = [int(x) for x in rng.choice(nq, k, replace=False)]
        mat = wl.haar_unitary(1 << k, rng)
        mask = sum(1 << t for t in targs)
        return (lambda h: qs.qs_apply_dense_block(h, targs, mat)), qs.QS_COST_FUSED_DENSE, k, mask, 0, 0
    if name in ("gate1", "dense"):
        n = 1 if name == "gate1" else int(rng.integers(2, 4))
        s = int(rng.integers(0, 4))
        qsel = [int(x) for x in rng.choice(nq, n + s, replace=False)]
        targs, ctrls = qsel[:n], qsel[n:]
        mat = wl.haar_unitary(1 << n, rng)
        mask = sum(1 << q for q in qsel)
        kind = qs.QS_COST_GATE1 if n == 1 else qs.QS_COST_DENSE
        return (lambda h: qs.qs_apply_ctrl_multi_target(h, ctrls, targs, mat)), kind, n, mask, s, 0
    if name == "diag":
        n = int(rng.integers(1, 4))
        targs = [int(x) for x in rng.choice(nq, n, replace=False)]
        d = np.exp(1j * rng.uniform(0, 2 * np.pi, 1 << n))
        return (lambda h: qs.qs_apply_diagonal(h, targs, d)), qs.QS_COST_DIAGONAL, n, sum(1 << t for t in targs), 0, 0
    w = int(rng.integers(1, 7))
    targs = [int(x) for x in rng.choice(nq, w, replace=False)]
    if name == "gadget":
        paulis = [int(x) for x in rng.integers(1, 4, size=w)]
        if not any(p in (1, 2) for p in paulis):
            paulis[0] = 1
        kind = qs.QS_COST_GADGET
    else:
        paulis = [3] * w
        kind = qs.QS_COST_PHASE
    theta = float(rng.uniform(0, 2 * np.pi))
    return (lambda h: qs.qs_apply_pauli_gadget(h, targs, paulis, theta)), kind, 0, sum(1 << t for t in targs), 0, w


def collect(samples, configs, seed=2311015122, device="cuda"):
    """Time `samples` random launches spread over configs = [(prec, qubits), ...].
    Returns (X [samples x 64] float32, t [samples] float32 = log ms, meta)."""
    import torch
    from . import qs
    rng = np.random.default_rng(seed)
    stream = torch.cuda.Stream()
    states = []
    for prec, nq in configs:
        dtype = torch.complex128 if prec == qs.QS_C128 else torch.complex64
        with torch.cuda.stream(stream):
            t = torch.randn(1 << nq, dtype=dtype, device=device)
            t /= torch.linalg.vector_norm(t)
        stream.synchronize()
        states.append((prec, nq, qs.State(nq, prec=prec, stream=stream, storage=t)))
    X = np.zeros((samples, 64), dtype=np.float32)
    y = np.zeros(samples, dtype=np.float32)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    # one warm-up launch of every kind on every state (first-launch costs)
    for _, nq, st in states:
        for _ in range(12):
            fn = _random_launch(qs, rng, nq)[0]
            fn(st.handle)
    stream.synchronize()
    t0 = time.time()
    for i in range(samples):
        prec, nq, st = states[i % len(states)]
        fn, kind, width, mask, nctrl, weight = _random_launch(qs, rng, nq)
        e0.record(stream)
        fn(st.handle)
        e1.record(stream)
        e1.synchronize()
        X[i] = qs.qs_costmodel_encode(kind, width, mask, nctrl, weight, st.handle)
        y[i] = math.log(max(e0.elapsed_time(e1), 1e-4))
    meta = {"samples": samples, "configs": configs, "seconds": time.time() - t0, "seed": seed}
    for _, _, st in states:
        st.close()
    return X, y, meta


def split(n, seed=7, validation=0.15, test=0.15):
    """Row indices of the training, validation (model selection) and test
    (reported only, never used for a choice) sets."""
    perm = np.random.default_rng(seed).permutation(n)
    nv, nt = int(n * validation), int(n * test)
    return perm[nv + nt:], perm[:nv], perm[nv:nv + nt]


def _errors(model, X, y):
    err = model.predict(X) - y
    return float(np.sqrt(np.mean(err ** 2))), float(np.median(np.abs(np.expm1(err))))


def train(X, y, epochs=300, batch=512, lr=2e-3, seed=7):
    """Train a fresh model on the GPU on the training rows; returns (model,
    metrics on the validation rows)."""
    from . import qs
    tr, va, _ = split(X.shape[0], seed)
    model = qs.CostModel(seed=seed)
    train_loss = model.train(X[tr], y[tr], epochs=epochs, batch=batch, lr=lr, seed=seed)
    rmse, med = _errors(model, X[va], y[va])
    metrics = {"train_mse_log": float(train_loss), "holdout_rmse_log": rmse,
               "holdout_median_abs_rel_time_error": med, "train_rows": int(len(tr)), "holdout_rows": int(len(va)),
               "holdout_role": "validation: chooses among the epoch settings"}
    return model, metrics


def save(model, path, meta):
    np.savez(path, params=model.get_params(), meta=json.dumps(meta))


def load(path=WEIGHTS_PATH):
    from . import qs
    data = np.load(path)
    model = qs.CostModel()
    model.set_params(data["params"])
    return model, json.loads(str(data["meta"]))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--samples", type=int, default=20000)
    ap.add_argument("--out", default=WEIGHTS_PATH)
    ap.add_argument("--epochs", type=int, nargs="+", default=[300],
                    help="train once per value; the model with the lowest validation error is saved and its "
                         "error on the separate test rows reported")
    ap.add_argument("--data-out", help="also save the timed rows (X, log ms) here")
    ap.add_argument("--data-in", help="train on rows saved by --data-out instead of timing new ones")
    args = ap.parse_args()
    if args.data_in:
        d = np.load(args.data_in)
        X, y, meta = d["X"], d["y"], json.loads(str(d["meta"]))
    else:
        configs = [(0, 24), (0, 27), (0, 30), (0, 32), (1, 24), (1, 27), (1, 30), (1, 31)]
        X, y, meta = collect(args.samples, configs)
        if args.data_out:
            np.savez(args.data_out, X=X, y=y, meta=json.dumps(meta))
    best = None
    for ep in args.epochs:
        model, metrics = train(X, y, epochs=ep)
        metrics["epochs"] = ep
        print(json.dumps(metrics), flush=True)
        if best is None or metrics["holdout_rmse_log"] < best[1]["holdout_rmse_log"]:
            if best is not None:
                best[0].close()
            best = (model, metrics)
        else:
            model.close()
    meta.update(best[1])
    # the test rows were used for nothing above: the reported error of the chosen model
    _, _, te = split(X.shape[0])
    rmse, med = _errors(best[0], X[te], y[te])
    meta.update({"test_rmse_log": rmse, "test_median_abs_rel_time_error": med, "test_rows": int(len(te))})
    save(best[0], args.out, meta)
    print(json.dumps(meta))


if __name__ == "__main__":
    main()
