"""Pins of the FP64 perceptron oracle: GELU against its erf definition and a
finite difference, the backward pass against central finite differences of
the loss, and Adam against its first-step closed form."""
import math

import numpy as np

from oracle import mlp as M


def test_gelu_definition_and_derivative():
    z = np.linspace(-4, 4, 41)
    ref = np.array([0.5 * t * (1 + math.erf(t / math.sqrt(2))) for t in z])
    np.testing.assert_allclose(M.gelu(z), ref, rtol=1e-15, atol=1e-16)
    h = 1e-6
    np.testing.assert_allclose(M.gelu_d(z), (M.gelu(z + h) - M.gelu(z - h)) / (2 * h), rtol=1e-8, atol=1e-9)
    assert abs(M.gelu(0.0)) == 0.0 and abs(M.gelu_d(0.0) - 0.5) < 1e-15


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(3)
    p = rng.normal(0, 0.3, M.NPARAMS)
    X = rng.normal(0, 1, (37, 3))
    Y = rng.normal(0, 1, (37, 4))
    loss, g = M.loss_grad(p, X, Y)
    assert loss > 0
    idx = rng.choice(M.NPARAMS, 60, replace=False)
    idx = np.concatenate([idx, [0, 191, 192, 255, 256, 4351, 4352, 4415, 4416, 4671, 4672, 4675]])
    for i in idx:
        e = np.zeros(M.NPARAMS)
        e[i] = 1e-6
        fd = (M.loss_grad(p + e, X, Y)[0] - M.loss_grad(p - e, X, Y)[0]) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g).max()), i


def test_layout_and_forward_by_loops():
    rng = np.random.default_rng(4)
    p = rng.normal(0, 0.2, M.NPARAMS)
    assert M.NPARAMS == 4676
    w = M.unpack(p)
    x = rng.normal(0, 1, 3)
    h1 = [M.gelu(sum(w["W1"][j, c] * x[c] for c in range(3)) + w["b1"][j]) for j in range(64)]
    h2 = [M.gelu(sum(w["W2"][j, i] * h1[i] for i in range(64)) + w["b2"][j]) for j in range(64)]
    y = [sum(w["W3"][k, j] * h2[j] for j in range(64)) + w["b3"][k] for k in range(4)]
    np.testing.assert_allclose(M.forward(p, x[None, :])[0][0], y, rtol=1e-12, atol=1e-14)


def test_adam_first_step_is_signed_lr():
    """With m = v = 0 and t = 1 the bias-corrected step is lr * g / (|g| + eps)."""
    g = np.array([0.3, -2.0, 1e-3])
    p1, m, v = M.adam(np.zeros(3), np.zeros(3), np.zeros(3), 1, g, lr=0.01)
    np.testing.assert_allclose(p1, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
