"""CPU oracle for the cost-model network (TEST INFRASTRUCTURE ONLY; see
qsim_oracle.py for who may import it).

The network predicts the log of a kernel's run time from a feature vector:
  h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = W3 h2 + b3,
with a mean-squared-error loss L = mean_b (y_b - t_b)^2 over a batch.  This is
the textbook two-hidden-layer perceptron; forward and backward are written out
here in float64 with plain numpy so that the GPU kernels' gradients can be
checked against them.  Pinned in tests/test_oracle_mlp.py by central finite
differences of the loss.

Parameter layout (shared with the CUDA kernels, as a flat float array):
  W1 [H x F] row-major, b1 [H], W2 [H x H], b2 [H], W3 [H], b3 [1].
"""

import numpy as np


def unpack(params, F, H):
    p = np.asarray(params, dtype=np.float64)
    o = 0
    W1 = p[o:o + H * F].reshape(H, F); o += H * F
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + H]; o += H
    b3 = p[o]; o += 1
    assert o == p.size
    return W1, b1, W2, b2, W3, b3


def num_params(F, H):
    return H * F + H + H * H + H + H + 1


def forward(params, X, F, H):
    """Predictions y [B] and the intermediates the backward pass needs."""
    W1, b1, W2, b2, W3, b3 = unpack(params, F, H)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3 + b3
    return y, (X, z1, h1, z2, h2)


def loss(params, X, t, F, H):
    y, _ = forward(params, X, F, H)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def backward(params, X, t, F, H):
    """Gradient of the mean-squared-error loss by the chain rule."""
    W1, b1, W2, b2, W3, b3 = unpack(params, F, H)
    y, (X, z1, h1, z2, h2) = forward(params, X, F, H)
    B = X.shape[0]
    dy = 2.0 * (y - np.asarray(t, dtype=np.float64)) / B      # dL/dy
    gW3 = h2.T @ dy
    gb3 = np.sum(dy)
    dh2 = np.outer(dy, W3)
    dz2 = dh2 * (z2 > 0)
    gW2 = dz2.T @ h1
    gb2 = np.sum(dz2, axis=0)
    dh1 = dz2 @ W2
    dz1 = dh1 * (z1 > 0)
    gW1 = dz1.T @ X
    gb1 = np.sum(dz1, axis=0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, [gb3]])


def adam_step(params, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """Adam (Kingma and Ba, 2015): bias-corrected first and second moments."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mhat = m / (1 - beta1 ** step)
    vhat = v / (1 - beta2 ** step)
    return params - lr * mhat / (np.sqrt(vhat) + eps), m, v
