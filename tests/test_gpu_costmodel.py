"""The fusion cost model: the GPU network's forward pass and gradient against
the float64 numpy oracle, training, and planning.  A plan must never change a
result, and on measured timings the learned plan must not lose to the plans
made without it."""

import numpy as np
import pytest

from oracle import mlp_oracle as mo
from oracle import qsim_oracle as orc
from paper_2311_01512_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
F = H = 64


@pytest.fixture(scope="module")
def qs():
    from paper_2311_01512_gb300 import qs as mod
    return mod


def test_forward_and_gradient_match_oracle(qs):
    rng = np.random.default_rng(5)
    params = (rng.standard_normal(qs.QS_COST_PARAMS) * 0.2).astype(np.float32)
    X = rng.standard_normal((96, F)).astype(np.float32)
    t = rng.standard_normal(96).astype(np.float32)
    m = qs.CostModel()
    m.set_params(params)
    y_gpu = m.predict(X)
    y_ref, _ = mo.forward(params.astype(np.float64), X, F, H)
    np.testing.assert_allclose(y_gpu, y_ref, rtol=1e-4, atol=1e-4)
    g_gpu, loss = m.gradient(X, t)
    g_ref = mo.backward(params.astype(np.float64), X, t, F, H)
    assert abs(loss - mo.loss(params, X, t, F, H)) <= 1e-4 * (1 + abs(loss))
    np.testing.assert_allclose(g_gpu, g_ref, rtol=2e-3, atol=2e-5 * float(np.max(np.abs(g_ref))))


def test_training_fits_a_smooth_target(qs):
    rng = np.random.default_rng(6)
    X = rng.random((4096, F)).astype(np.float32)
    w = rng.standard_normal(F)
    t = (np.log1p(np.exp(X @ w)) + 0.3 * X[:, 0] * X[:, 1]).astype(np.float32)
    m = qs.CostModel(seed=3)
    _, loss0 = m.gradient(X, t)
    loss = m.train(X, t, epochs=60, batch=256, lr=2e-3)
    assert loss < 0.05 * loss0, (loss, loss0)


def test_cost_plan_keeps_results(qs):
    rng = wl.rng_for("costplan-results")
    nq = 11
    psi = wl.random_statevector(nq, rng)
    ops = wl.statevector_circuit(nq, 120, rng, max_targs=3, max_ctrls=2)
    want = orc.run_ops(psi, ops, is_density=False)
    st = qs.State(nq)
    st.set_amps(psi)
    model = qs.CostModel(seed=11)                 # untrained: any plan must be exact
    circ = qs.Circuit(nq, ops)
    circ.plan_cost(model, st.handle, max_block_qubits=4, window=16)
    circ.apply(st.handle)
    assert float(np.max(np.abs(st.get_amps() - want))) <= 0.3e-12


def _time_plan(qs, torch, circ, st, reps=3):
    best = 1e30
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st.stream)
        circ.apply(st.handle)
        e1.record(st.stream)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def test_learned_plan_beats_plans_without_it(qs):
    """A/B on measured time: the cost-model plan against no fusion and greedy
    fusion, on a 400-gate circuit of the fused workload's mix (26-qubit
    complex64 state; the model is trained here on 3000 timings)."""
    import torch
    from paper_2311_01512_gb300 import costmodel
    nq = 26
    X, y, _ = costmodel.collect(3000, [(0, nq)], seed=99)
    model, metrics = costmodel.train(X, y, epochs=120)
    assert metrics["holdout_rmse_log"] < 0.6
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        t = torch.randn(1 << nq, dtype=torch.complex64, device="cuda")
        t /= torch.linalg.vector_norm(t)
    stream.synchronize()
    st = qs.State(nq, prec=0, stream=stream, storage=t)
    ops = wl.unitary_circuit(nq, 400, wl.rng_for("ab-circuit"))
    times = {}
    for name in ("none", "greedy3", "greedy5", "cost"):
        circ = qs.Circuit(nq, ops)
        if name == "none":
            circ.plan(qs.QS_PLAN_NONE, 1)
        elif name.startswith("greedy"):
            circ.plan(qs.QS_PLAN_GREEDY, int(name[-1]))
        else:
            circ.plan_cost(model, st.handle, max_block_qubits=5, window=24)
        circ.apply(st.handle)                     # warm-up
        times[name] = _time_plan(qs, torch, circ, st)
        circ.close()
    print("plan times (ms):", times)
    assert times["cost"] <= 1.05 * min(times["none"], times["greedy3"], times["greedy5"]), times
