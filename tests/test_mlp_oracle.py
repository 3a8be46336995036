"""Pins of the surrogate-network oracle (FP64, CPU)."""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as M


def test_gelu_closed_form_values():
    # GELU(z) = z Phi(z); Phi(1) = 0.8413447460685429 (standard normal table)
    assert M.gelu(np.array([0.0]))[0] == 0.0
    assert M.gelu(np.array([1.0]))[0] == pytest.approx(0.8413447460685429, rel=1e-15)
    assert M.gelu(np.array([-1.0]))[0] == pytest.approx(-(1 - 0.8413447460685429), rel=1e-14)
    assert M.gelu(np.array([10.0]))[0] == pytest.approx(10.0, rel=1e-15)
    assert M.gelu_grad(np.array([0.0]))[0] == 0.5
    z = np.linspace(-4, 4, 17)
    h = 1e-6
    fd = (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)
    assert np.allclose(M.gelu_grad(z), fd, rtol=1e-8, atol=1e-10)


def test_bf16_rounding_is_round_to_nearest_even():
    x = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -7, -(1 + 2 ** -8 + 2 ** -12), 3.0e-3, 0.0])
    want = np.array([1.0, 1.0, 1 + 2 ** -6, 1 + 2 ** -7, -(1 + 2 ** -7), None, 0.0], dtype=object)
    got = M.round_bf16(x)
    for g, w in zip(got, want):
        if w is not None:
            assert g == w
    # 8 significant bits: relative rounding error at most half an ulp, 2^-8
    r = np.random.default_rng(0).uniform(-100, 100, 1000)
    assert np.all(np.abs(M.round_bf16(r) - r) <= 2 ** -8 * np.abs(r))


def test_single_path_network_is_a_gelu_composition():
    th = np.zeros(M.n_params())
    (W1, b1), (W2, b2), (W3, b3), (W4, b4) = M.unpack(th)
    W1[0, 0] = W2[0, 0] = W3[0, 0] = W4[0, 0] = 1.0
    b4[1] = 0.25
    x = np.array([[0.7, 1, 2, 3, 4, 5]])
    y, _ = M.forward(th, x)

    def g(v):
        return v * 0.5 * (1 + math.erf(v / math.sqrt(2)))
    assert y[0, 0] == pytest.approx(g(g(g(0.7))), rel=1e-14)
    assert y[0, 1] == 0.25 and y[0, 2] == 0.0


def test_zero_weights_give_output_bias():
    th = M.init_params(1)
    for W, b in M.unpack(th):
        W[:] = 0.0
        b[:] = 0.3
    y, _ = M.forward(th, np.random.default_rng(0).normal(size=(5, 6)))
    assert np.all(y == 0.3)


def test_backward_matches_central_differences():
    rng = np.random.default_rng(3)
    th = M.init_params(7)
    X = rng.normal(size=(9, 6))
    T = rng.normal(size=(9, 3))
    _, g = M.backward(th, X, T)
    idx = rng.choice(th.size, 60, replace=False)
    idx = np.concatenate([idx, [th.size - 1, th.size - 4, 6 * 128 + 5]])   # biases of the last/first layer
    h = 1e-6
    for i in idx:
        e = np.zeros_like(th)
        e[i] = h
        fd = (M.loss(th + e, X, T) - M.loss(th - e, X, T)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-10)


def test_adam_first_step_is_signed_learning_rate():
    th = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -1e-3, 2.0])
    new, m, v = M.adam(th, np.zeros(3), np.zeros(3), g, 1, 1e-2)
    assert np.allclose(new, th - 1e-2 * np.sign(g), rtol=0, atol=1e-7)


def test_training_reduces_the_loss():
    rng = np.random.default_rng(5)
    X = rng.uniform(-1, 1, size=(64, 6))
    T = np.stack([np.sin(X[:, 0]), X[:, 1] * X[:, 2], np.cos(X[:, 3])], axis=1)
    th = M.init_params(2)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    l0 = M.loss(th, X, T)
    for s in range(1, 151):
        _, g = M.backward(th, X, T)
        th, m, v = M.adam(th, m, v, g, s, 3e-3)
    assert M.loss(th, X, T) < 0.2 * l0
