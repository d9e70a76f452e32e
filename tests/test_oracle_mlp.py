"""Pins for the cost-model network oracle (oracle/mlp_oracle.py): the
backward pass against central finite differences of the loss, a forward pass
worked by hand, and the first Adam step's closed form.  CPU only."""

import numpy as np

from oracle import mlp_oracle as mo


def test_forward_by_hand():
    F, H = 2, 2
    W1 = np.array([[1.0, -1.0], [0.5, 2.0]]); b1 = np.array([0.0, -1.0])
    W2 = np.array([[1.0, 1.0], [-1.0, 0.0]]); b2 = np.array([0.5, 0.0])
    W3 = np.array([2.0, 3.0]); b3 = -1.0
    params = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3, [b3]])
    x = np.array([[1.0, 2.0]])
    # z1 = [1 - 2, 0.5 + 4 - 1] = [-1, 3.5] -> h1 = [0, 3.5]
    # z2 = [0 + 3.5 + 0.5, 0] = [4, 0] -> h2 = [4, 0]; y = 8 - 1 = 7
    y, _ = mo.forward(params, x, F, H)
    assert y[0] == 7.0


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    F, H, B = 7, 5, 11
    params = rng.standard_normal(mo.num_params(F, H)) * 0.7
    X = rng.standard_normal((B, F))
    t = rng.standard_normal(B)
    g = mo.backward(params, X, t, F, H)
    eps = 1e-6
    fd = np.empty_like(params)
    for i in range(params.size):
        p1 = params.copy(); p1[i] += eps
        p2 = params.copy(); p2[i] -= eps
        fd[i] = (mo.loss(p1, X, t, F, H) - mo.loss(p2, X, t, F, H)) / (2 * eps)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-8)


def test_first_adam_step_is_sign_step():
    p = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -4.0, 1e-3])
    new, m, v = mo.adam_step(p, g, np.zeros(3), np.zeros(3), 1, lr=0.1)
    # bias-corrected moments at step 1 are g and g^2: the step is lr * g / (|g| + eps)
    np.testing.assert_allclose(new, p - 0.1 * g / (np.abs(g) + 1e-8), rtol=1e-12)
