"""Pins of the MLP oracle: backward against central finite differences (in
FP64, rounding off), bf16 rounding against its definition, and a descent
step that lowers the loss.  No GPU."""

import numpy as np
import pytest

from oracle import mlp


def _data(n=64, f=8, seed=0):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, f))
    t = rng.standard_normal(n)
    return x, t


def test_backward_matches_finite_differences():
    x, t = _data()
    theta = mlp.init_params(x.shape[1], 3).astype(np.float64)
    theta[:] += 0.01 * np.random.default_rng(4).standard_normal(theta.size)  # nonzero biases
    _, g = mlp.loss_and_grad(theta, x, t, round_bf16=False)
    h = 1e-6
    rng = np.random.default_rng(5)
    for i in rng.choice(theta.size, 60, replace=False):
        tp = theta.copy()
        tm = theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss_and_grad(tp, x, t, round_bf16=False)[0] -
              mlp.loss_and_grad(tm, x, t, round_bf16=False)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-8)


def test_bf16_round_definition():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 3.14159, -2.71828, 1e-30, 0.0], np.float32)
    r = mlp.bf16_round(vals)
    for v, rv in zip(vals, r):
        # bfloat16 keeps 8 significant bits: the rounded value is the nearest
        # multiple of 2^(e-7), e = floor(log2|v|)
        if v == 0:
            assert rv == 0
            continue
        e = np.floor(np.log2(abs(float(v))))
        q = 2.0 ** (e - 7)
        assert abs(rv - float(v)) <= q / 2 + 1e-45
        assert abs(rv / q - round(rv / q)) < 1e-9
    assert r[1] == 1.0  # exact tie rounds to even
    assert r[2] == 1.0 + 2 ** -7


def test_adam_step_lowers_loss():
    x, t = _data(256)
    theta = mlp.init_params(x.shape[1], 7)
    m = np.zeros(theta.size)
    v = np.zeros(theta.size)
    l0, _ = mlp.loss_and_grad(theta, x, t)
    for step in range(1, 51):
        _, g = mlp.loss_and_grad(theta, x, t)
        theta, m, v = mlp.adam_step(theta, g, m, v, step, 1e-2)
    l1, _ = mlp.loss_and_grad(theta, x, t)
    assert l1 < 0.7 * l0
