"""Pins of the cost-model MLP oracle (F -> H -> H -> 1, ReLU, MSE, Adam)."""
import numpy as np
import pytest

import oracle
import synth


def make_params(F, H, seed=7, scale=0.5):
    v = synth.uniform_np(seed, 0, H * F + H + H * H + H + H + 1) * scale
    return oracle.MLPParams.from_flat(v, F, H)


def test_central_finite_differences():
    F, H, B = 5, 8, 11
    p = make_params(F, H)
    X = synth.uniform_np(8, 0, B * F).reshape(B, F)
    t = synth.uniform_np(9, 0, B)
    loss, g = oracle.mlp_loss_grad(p, X, t)
    theta = p.flat()
    gflat = g.flat()
    h = 1e-6
    rng_idx = list(range(0, theta.size, 3))
    for i in rng_idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        lp, _ = oracle.mlp_loss_grad(oracle.MLPParams.from_flat(tp, F, H), X, t)
        lm, _ = oracle.mlp_loss_grad(oracle.MLPParams.from_flat(tm, F, H), X, t)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gflat[i]) <= 1e-6 * max(1.0, abs(gflat[i])), i


def test_forward_matches_loss_path():
    F, H, B = 7, 16, 9
    p = make_params(F, H)
    X = synth.uniform_np(3, 0, B * F).reshape(B, F)
    y, h1, h2 = oracle.mlp_forward(p, X)
    t = y.copy()
    loss, g = oracle.mlp_loss_grad(p, X, t)
    assert loss == 0.0
    assert np.all(g.flat() == 0.0)
    assert np.all(h1 >= 0) and np.all(h2 >= 0)


def test_linear_regime_matches_least_squares_gradient():
    """All pre-activations positive => the net is affine; gradients have a
    closed form through ordinary matrix products (numpy, not the oracle)."""
    F, H, B = 4, 6, 10
    rng = np.random.default_rng(3)
    W1 = rng.uniform(0.1, 0.5, (H, F)); b1 = rng.uniform(1.0, 2.0, H)
    W2 = rng.uniform(0.1, 0.5, (H, H)); b2 = rng.uniform(1.0, 2.0, H)
    w3 = rng.uniform(-1, 1, H); b3 = np.array([0.3])
    X = rng.uniform(0.0, 1.0, (B, F))
    t = rng.uniform(-1, 1, B)
    p = oracle.MLPParams(W1, b1, W2, b2, w3, b3)
    loss, g = oracle.mlp_loss_grad(p, X, t)
    H1 = X @ W1.T + b1
    H2 = H1 @ W2.T + b2
    y = H2 @ w3 + b3[0]
    r = y - t
    dy = 2 * r / B
    np.testing.assert_allclose(loss, np.mean(r ** 2), rtol=1e-13)
    np.testing.assert_allclose(g.b3[0], dy.sum(), rtol=1e-12)
    np.testing.assert_allclose(g.w3, H2.T @ dy, rtol=1e-12)
    D2 = np.outer(dy, w3)
    np.testing.assert_allclose(g.W2, D2.T @ H1, rtol=1e-12)
    np.testing.assert_allclose(g.b2, D2.sum(0), rtol=1e-12)
    D1 = D2 @ W2
    np.testing.assert_allclose(g.W1, D1.T @ X, rtol=1e-12)
    np.testing.assert_allclose(g.b1, D1.sum(0), rtol=1e-12)


def test_relu_kink_has_zero_gradient():
    F, H = 2, 3
    p = oracle.MLPParams(np.zeros((H, F)), np.zeros(H), np.eye(H), np.zeros(H), np.ones(H), np.zeros(1))
    _, g = oracle.mlp_loss_grad(p, np.ones((1, F)), np.array([1.0]))
    assert np.all(g.W1 == 0) and np.all(g.W2 == 0)


@pytest.mark.parametrize("steps", [1, 5])
def test_adam_constant_gradient_closed_form(steps):
    """With a constant gradient g, bias-corrected moments are exactly g and
    g^2, so every step moves theta by lr * g / (|g| + eps)."""
    gvec = np.array([0.5, -2.0, 1e-3, 3.0])
    theta = np.array([1.0, 2.0, 3.0, 4.0])
    m = np.zeros(4); v = np.zeros(4)
    th = theta.copy()
    for s in range(1, steps + 1):
        oracle.adam(th, gvec.copy(), m, v, s, lr=1e-2)
    expect = theta - steps * 1e-2 * gvec / (np.abs(gvec) + 1e-8)
    np.testing.assert_allclose(th, expect, rtol=1e-12, atol=1e-12)
