"""FP64 oracle of the per-coordinate MLP used by the learned warm start and
preconditioner -- TEST INFRASTRUCTURE ONLY.

The paper has no learned component; this follows the design of the
library's learned path (features, network, loss, optimiser), written out
plainly in float64 so the GPU kernels can be checked against it.

Features of coordinate d at E-step t (before the solve), with the Jacobi
diagonal of A, c_d = beta ||phi_d||^2 + alpha_d:
    u1 = ln(alpha_d) / 10
    u2 = ln(beta ||phi_d||^2) / 10
    u3 = asinh(mu_prev_d * sqrt(c_d)) / 4
    u4 = ln(max(s_prev_d * c_d, 1e-6)) / 4
Targets (the same transforms of the E-step's own mu and s):
    y1 = asinh(mu_d * sqrt(c_d)) / 4,   y2 = ln(max(s_d * c_d, 1e-6)) / 4
Network (1282 parameters): a1 = W1 u + b1, h1 = tanh(a1), a2 = W2 h1 + b2,
h2 = tanh(a2), o = W3 h2 + b3 with W1 32x4, W2 32x32, W3 2x32.
Loss: mean over samples of 1/2 ||o - y||^2.  Optimiser: Adam.
Predictions: mu_hat = sinh(4 o1) / sqrt(c_d),  s_hat = exp(4 clip(o2)) / c_d.

Parity status: forward/backward pinned by central finite differences and by
closed forms of degenerate networks (tests/test_oracle_mlp.py).
"""
import numpy as np

SHAPES = [("W1", (32, 4)), ("b1", (32,)), ("W2", (32, 32)), ("b2", (32,)),
          ("W3", (2, 32)), ("b3", (2,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)      # 1282


def unpack(theta):
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = theta[o:o + n].reshape(shp)
        o += n
    return out


def init_params(seed):
    """Glorot-uniform weights, zero biases (float64 vector of 1282)."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shp in SHAPES:
        if name.startswith("W"):
            lim = np.sqrt(6.0 / (shp[0] + shp[1]))
            parts.append(rng.uniform(-lim, lim, size=shp).ravel())
        else:
            parts.append(np.zeros(shp))
    return np.concatenate(parts)


def features(alpha, phi_norm2, beta, mu_prev, s_prev):
    c = beta * phi_norm2 + alpha
    return np.stack([np.log(alpha) / 10.0, np.log(beta * phi_norm2) / 10.0,
                     np.arcsinh(mu_prev * np.sqrt(c)) / 4.0,
                     np.log(np.maximum(s_prev * c, 1e-6)) / 4.0], axis=1)


def targets(alpha, phi_norm2, beta, mu, s):
    c = beta * phi_norm2 + alpha
    return np.stack([np.arcsinh(mu * np.sqrt(c)) / 4.0,
                     np.log(np.maximum(s * c, 1e-6)) / 4.0], axis=1)


def predict(o, alpha, phi_norm2, beta):
    """(mu_hat, s_hat) from network outputs o (n x 2)."""
    c = beta * phi_norm2 + alpha
    return np.sinh(4.0 * o[:, 0]) / np.sqrt(c), np.exp(4.0 * np.clip(o[:, 1], -10, 10)) / c


def forward(theta, U):
    p = unpack(theta)
    a1 = U @ p["W1"].T + p["b1"]
    h1 = np.tanh(a1)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.tanh(a2)
    o = h2 @ p["W3"].T + p["b3"]
    return o, (U, h1, h2)


def loss(theta, U, Y):
    o, _ = forward(theta, U)
    return 0.5 * np.mean(np.sum((o - Y) ** 2, axis=1))


def grad(theta, U, Y):
    """Gradient of loss(theta, U, Y) by backpropagation (same layout as theta)."""
    p = unpack(theta)
    o, (U, h1, h2) = forward(theta, U)
    n = U.shape[0]
    go = (o - Y) / n
    gW3 = go.T @ h2
    gb3 = go.sum(axis=0)
    gh2 = go @ p["W3"]
    ga2 = gh2 * (1.0 - h2 ** 2)
    gW2 = ga2.T @ h1
    gb2 = ga2.sum(axis=0)
    gh1 = ga2 @ p["W2"]
    ga1 = gh1 * (1.0 - h1 ** 2)
    gW1 = ga1.T @ U
    gb1 = ga1.sum(axis=0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])


def adam_step(theta, g, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba); step is 1-based.  Returns (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
