"""Pins of the FP64 reference of the learned-guess network (closed forms,
adjoint identities, finite differences)."""
import math

import numpy as np
import pytest

from oracle import cnn_oracle as C
from paper_1703_01202_gb300 import inputs


def test_param_count():
    assert C.param_count() == 3 * 32 * 9 + 32 + 2 * (32 * 32 * 9 + 32) + 32 * 9 + 1 == 19681


def test_conv_of_a_delta_is_the_kernel():
    rng = np.random.default_rng(1)
    w = rng.normal(size=(4, 2, 3, 3))
    b = rng.normal(size=4)
    x = np.zeros((2, 7, 9))
    x[1, 3, 5] = 1.0
    out = C.conv3x3(x, w, b)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):  # out[y, x] reads x[y + dy, x + dx]
            np.testing.assert_allclose(out[:, 3 - dy, 5 - dx], b + w[:, 1, dy + 1, dx + 1], rtol=1e-14)
    # periodic wrap: a delta in the corner reaches the opposite corner
    x = np.zeros((2, 7, 9))
    x[0, 0, 0] = 1.0
    np.testing.assert_allclose(C.conv3x3(x, w, b)[:, 6, 8], b + w[:, 0, 2, 2], rtol=1e-14)


def test_conv_adjoints():
    rng = np.random.default_rng(2)
    w = rng.normal(size=(5, 3, 3, 3))
    b = np.zeros(5)
    x = rng.normal(size=(3, 8, 6))
    y = rng.normal(size=(5, 8, 6))
    lhs = np.sum(C.conv3x3(x, w, b) * y)
    assert lhs == pytest.approx(np.sum(x * C.conv3x3_grad_input(y, w)), rel=1e-12)
    dw, db = C.conv3x3_grad_weight(x, y)
    assert lhs == pytest.approx(np.sum(w * dw), rel=1e-12)
    np.testing.assert_allclose(db, y.sum(axis=(1, 2)), rtol=1e-14)


def test_gelu_closed_forms():
    assert C.gelu(np.array([0.0]))[0] == 0.0
    x = np.linspace(-4, 4, 33)
    np.testing.assert_allclose(C.gelu(x) - C.gelu(-x), x, atol=1e-15)  # x Phi(x) + x Phi(x) - x
    assert C.gelu(np.array([10.0]))[0] == pytest.approx(10.0, rel=1e-15)
    h = 1e-6
    np.testing.assert_allclose(C.gelu_grad(x), (C.gelu(x + h) - C.gelu(x - h)) / (2 * h), rtol=1e-8, atol=1e-9)


def test_loss_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    theta = C.init_params(4)
    theta[-(32 * 9 + 1):] = rng.normal(scale=0.2, size=32 * 9 + 1)  # non-trivial last layer
    inp = rng.normal(size=(3, 10, 12))
    tgt = rng.normal(size=(10, 12))
    loss, g = C.loss_and_grad(theta, inp, tgt)
    idx = rng.choice(theta.size, 8, replace=False)
    for i in idx:
        e = np.zeros_like(theta)
        h = 1e-5 * max(1.0, abs(theta[i]))
        e[i] = h
        fd = (C.loss_and_grad(theta + e, inp, tgt)[0] - C.loss_and_grad(theta - e, inp, tgt)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-10)


def test_adam_first_step_is_a_signed_step():
    g = np.array([0.5, -2.0, 1e-3])
    th, m, v = C.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    np.testing.assert_allclose(th, -0.01 * np.sign(g), rtol=1e-5)


def test_guess_keeps_mass_and_reduces_to_extrapolation():
    shape = (16, 20)
    phin = inputs.noise_field(shape, 0.2, 0.1, 1)
    phinm1 = inputs.noise_field(shape, 0.2, 0.1, 2)
    phinm1 += phin.mean() - phinm1.mean()
    theta = np.zeros(C.param_count())
    g = C.guess(theta, phin, phinm1, 2.0, 1.0, 10.0, 0.01)
    np.testing.assert_allclose(g, phin + 2.0 * (phin - phinm1), atol=1e-14)
    theta = C.init_params(5)
    g = C.guess(theta, phin, phinm1, 2.0, 1.0, 10.0, 0.01)
    assert g.mean() == pytest.approx(phin.mean(), abs=1e-15)
