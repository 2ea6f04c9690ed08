"""Pins of the oracle MLP (learned warm start / preconditioner): gradients
by central finite differences, closed forms of degenerate networks, and
Adam's first step.  CPU only."""
import numpy as np

from oracle import mlp


def _data(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, 4)), rng.standard_normal((n, 2))


def test_param_count():
    assert mlp.N_PARAMS == 1282


def test_gradient_matches_central_differences():
    theta = mlp.init_params(0) + 0.05 * np.random.default_rng(1).standard_normal(mlp.N_PARAMS)
    U, Y = _data(37, 2)
    g = mlp.grad(theta, U, Y)
    h = 1e-6
    idx = np.random.default_rng(3).choice(mlp.N_PARAMS, size=120, replace=False)
    for i in idx:
        e = np.zeros(mlp.N_PARAMS)
        e[i] = h
        fd = (mlp.loss(theta + e, U, Y) - mlp.loss(theta - e, U, Y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)), i


def test_linear_regime_closed_form():
    # with W1 = W2 = 0 the hidden layers are constant tanh(b); o = W3 h2 + b3,
    # and the loss gradient in b3 is mean(o - y)
    theta = np.zeros(mlp.N_PARAMS)
    p = mlp.unpack(theta)
    p["b1"][:] = 0.3
    p["b2"][:] = -0.2
    p["W3"][:] = 0.5
    p["b3"][:] = [0.1, -0.4]
    U, Y = _data(50, 4)
    o, _ = mlp.forward(theta, U)
    h2 = np.tanh(-0.2) * np.ones(32)
    np.testing.assert_allclose(o, np.tile(0.5 * h2.sum() + np.array([0.1, -0.4]), (50, 1)),
                               rtol=1e-14)
    g = mlp.unpack(mlp.grad(theta, U, Y))
    np.testing.assert_allclose(g["b3"], (o - Y).mean(axis=0), rtol=1e-14)
    assert np.all(g["W1"] == 0)        # no signal reaches W1 when W2 = 0


def test_adam_first_step_moves_by_lr():
    theta = np.zeros(5)
    g = np.array([1e-3, -2.0, 0.5, 0.0, 7.0])
    t1, m, v = mlp.adam_step(theta, g, np.zeros(5), np.zeros(5), 1, lr=0.01)
    # bias-corrected first step is lr * sign(g) (up to eps)
    np.testing.assert_allclose(t1[[0, 1, 2, 4]], -0.01 * np.sign(g[[0, 1, 2, 4]]), rtol=1e-4)
    assert t1[3] == 0


def test_features_targets_roundtrip():
    rng = np.random.default_rng(5)
    alpha = np.exp(rng.uniform(-2, 20, 100))
    pn = rng.uniform(0.5, 2, 100)
    beta = 1e4
    mu = rng.standard_normal(100) * 1e-2
    s = 1.0 / (beta * pn + alpha) * np.exp(rng.uniform(-1, 1, 100))
    Y = mlp.targets(alpha, pn, beta, mu, s)
    mu_hat, s_hat = mlp.predict(Y, alpha, pn, beta)
    np.testing.assert_allclose(mu_hat, mu, rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(s_hat, s, rtol=1e-12)
    F = mlp.features(alpha, pn, beta, mu, s)
    np.testing.assert_allclose(F[:, 2:], Y, rtol=1e-14)     # previous-step features = targets
