"""Oracle for the learned block-norm predictor (not in the paper: a learned
skip of tasks on top of the exact block filter).  FP64 numpy forward and backward of a
2-hidden-layer ReLU network whose weights are rounded to bfloat16 before use
(the GPU keeps FP32 master weights and multiplies with their bf16 copies,
accumulating in FP32), with a mean-squared-error loss on log10 norms.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Parameters, in the flat order shared with the library:
    W1 [H][F], b1 [H], W2 [H][H], b2 [H], w3 [H], b3 [1]
Forward:   z1 = W1 x + b1, h1 = relu(z1), z2 = W2 h1 + b2, h2 = relu(z2),
           y = w3 . h2 + b3 + x[BOUND]
(the last feature is log10 of the norm-product bound of a task; the network
learns the residual, log10 of actual norm / bound, which is <= 0)
Loss:      L = mean_s (y_s - t_s)^2
Gradients are taken with respect to the bf16-rounded weights and applied to
the master weights (straight-through rounding).
"""

from __future__ import annotations

import numpy as np

HIDDEN = 64
BOUND = 7  # index of the log10 norm-product bound among the features


def n_params(n_feat: int, hidden: int = HIDDEN) -> int:
    return hidden * n_feat + hidden + hidden * hidden + hidden + hidden + 1


def unpack(theta: np.ndarray, n_feat: int, hidden: int = HIDDEN):
    i = 0
    out = []
    for shape in ((hidden, n_feat), (hidden,), (hidden, hidden), (hidden,), (hidden,), (1,)):
        k = int(np.prod(shape))
        out.append(theta[i:i + k].reshape(shape))
        i += k
    return out


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even)."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(theta: np.ndarray, x: np.ndarray, hidden: int = HIDDEN, round_bf16: bool = True):
    n_feat = x.shape[1]
    th = bf16_round(theta) if round_bf16 else theta.astype(np.float64)
    w1, b1, w2, b2, w3, b3 = unpack(th, n_feat, hidden)
    z1 = x @ w1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ w2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w3 + b3[0] + x[:, BOUND]
    return y, (z1, h1, z2, h2, th)


def loss_and_grad(theta: np.ndarray, x: np.ndarray, t: np.ndarray, hidden: int = HIDDEN,
                  round_bf16: bool = True):
    """(L, dL/dtheta) by the chain rule, layer by layer."""
    n, n_feat = x.shape
    y, (z1, h1, z2, h2, th) = forward(theta, x, hidden, round_bf16)
    w1, b1, w2, b2, w3, b3 = unpack(th, n_feat, hidden)
    r = y - t
    loss = float(np.mean(r * r))
    dy = 2.0 * r / n                       # [n]
    dw3 = h2.T @ dy
    db3 = np.array([dy.sum()])
    dh2 = np.outer(dy, w3)
    dz2 = dh2 * (z2 > 0.0)
    dw2 = dz2.T @ h1
    db2 = dz2.sum(axis=0)
    dh1 = dz2 @ w2
    dz1 = dh1 * (z1 > 0.0)
    dw1 = dz1.T @ x
    db1 = dz1.sum(axis=0)
    grad = np.concatenate([dw1.ravel(), db1, dw2.ravel(), db2, dw3, db3])
    return loss, grad


def init_params(n_feat: int, seed: int, hidden: int = HIDDEN) -> np.ndarray:
    """He-style initial weights from a seeded generator, zero biases."""
    rng = np.random.default_rng(seed)
    w1 = rng.standard_normal((hidden, n_feat)) * np.sqrt(2.0 / n_feat)
    w2 = rng.standard_normal((hidden, hidden)) * np.sqrt(2.0 / hidden)
    w3 = rng.standard_normal(hidden) * np.sqrt(1.0 / hidden)
    return np.concatenate([w1.ravel(), np.zeros(hidden), w2.ravel(), np.zeros(hidden), w3,
                           np.zeros(1)]).astype(np.float32)


def adam_step(theta, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) of FP32 master weights."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return (theta - lr * mh / (np.sqrt(vh) + eps)).astype(np.float32), m, v
