"""Pins for the network oracle: gradients against central finite
differences, the stable loss against its naive form, the first Adam step in
closed form, the monotone choice rule, and features on hand-made inputs."""
import math

import numpy as np

from oracle import mlp


def _rand(seed, batch=7):
    rng = np.random.default_rng(seed)
    theta = rng.standard_normal(mlp.n_params()) * 0.3
    X = rng.standard_normal((batch, mlp.N_IN))
    Y = (rng.random((batch, mlp.N_OUT)) > 0.5).astype(float)
    return theta, X, Y


def test_param_count():
    assert mlp.n_params() == 64 * 39 + 64 + 64 * 64 + 64 + 21 * 64 + 21
    theta = np.arange(mlp.n_params(), dtype=float)
    assert np.array_equal(mlp.pack(mlp.unpack(theta)), theta)


def test_backward_matches_finite_differences():
    theta, X, Y = _rand(1)
    z, cache = mlp.forward(theta, X)
    g = mlp.backward(theta, cache, z, Y)
    rng = np.random.default_rng(2)
    idx = rng.choice(mlp.n_params(), 60, replace=False)
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        num = (mlp.loss(mlp.forward(tp, X)[0], Y) - mlp.loss(mlp.forward(tm, X)[0], Y)) / (2 * h)
        assert abs(num - g[i]) <= 1e-7 + 1e-5 * abs(num), (i, num, g[i])


def test_stable_loss_equals_naive():
    rng = np.random.default_rng(3)
    z = rng.standard_normal((5, 21)) * 4
    Y = (rng.random((5, 21)) > 0.3).astype(float)
    s = 1 / (1 + np.exp(-z))
    naive = -(Y * np.log(s) + (1 - Y) * np.log(1 - s)).sum() / 5
    assert abs(mlp.loss(z, Y) - naive) < 1e-12


def test_first_adam_step_closed_form():
    # t = 1: m_hat = g, v_hat = g^2, so each parameter moves by lr * g / (|g| + eps)
    rng = np.random.default_rng(4)
    theta = rng.standard_normal(50)
    g = rng.standard_normal(50)
    th1, m, v = mlp.adam_step(theta, g, np.zeros(50), np.zeros(50), 1, lr=0.01)
    assert np.allclose(th1, theta - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_choose_rule():
    z = np.full(21, 10.0)
    assert mlp.choose(z) == 4
    z[:6] = -10.0                     # N = 4..9 fail
    assert mlp.choose(z) == 10
    z[12] = -10.0                     # N = 16 fails: only 17.. qualify
    assert mlp.choose(z) == 17
    assert mlp.choose(np.full(21, -5.0)) is None


def test_features_closed_forms():
    # one row: 1, 0.5, 0.25, 0 (real), imaginary all zero -> spans 0, 1, 2 and five zeros
    A = np.array([[1.0, 0.5, 0.25, 0.0]], dtype=complex)
    B = np.ones((4, 2), dtype=complex) * (1 + 1j)
    f = mlp.features(A, B, 1e-10)
    assert np.allclose(f[0:3], [1 / 8, 1 / 8, 1 / 8]) and math.isclose(f[15], 5 / 8)
    # B: all entries equal -> span 0 for all 8 per column, t = 1 -> S = 8 * 2^30, L = 0.5 log2(8)
    assert math.isclose(f[16], 1.0) and math.isclose(f[34], 1.5) and math.isclose(f[35], 1.5)
    assert math.isclose(f[36], 2 / 17) and math.isclose(f[37], 10 / 16) and f[38] == 0.0
    # A row: t = 1, 0.5, 0.25 -> ceil(t 2^15)^2 sums to 2^30 (1 + 1/4 + 1/16)
    La = 0.5 * math.log2(1 + 0.25 + 0.0625)
    assert math.isclose(f[32], La) and math.isclose(f[33], La)


def test_forward_closed_form():
    """Hand-set weights whose logits follow by hand: hidden unit 0 copies
    feature 3, hidden unit 1 copies -feature 5 (so the ReLU passes one sign
    only), layer 2 sums them with weights 2 and -3 into unit 7, and output t
    reads unit 7 with weight t and bias -t."""
    W1 = np.zeros((64, 39))
    b1 = np.zeros(64)
    W2 = np.zeros((64, 64))
    b2 = np.zeros(64)
    W3 = np.zeros((21, 64))
    b3 = np.zeros(21)
    W1[0, 3] = 1.0
    W1[1, 5] = -1.0
    b1[2] = -1.0                          # a unit the ReLU always zeroes
    W2[7, 0], W2[7, 1], W2[7, 2] = 2.0, -3.0, 100.0
    b2[7] = 0.5
    for t in range(21):
        W3[t, 7] = float(t)
        b3[t] = -float(t)
    theta = mlp.pack([W1, b1, W2, b2, W3, b3])
    X = np.zeros((4, 39))
    X[0, 3], X[0, 5] = 1.5, -2.0          # h1 = (1.5, 2.0): a2 = 3 - 6 + 0.5 = -2.5 -> 0
    X[1, 3], X[1, 5] = 4.0, 1.0           # h1 = (4, 0): a2 = 8.5
    X[2, 3], X[2, 5] = -1.0, -0.25        # h1 = (0, 0.25): a2 = -0.75 + 0.5 = -0.25 -> 0
    X[3, 3], X[3, 5] = 0.25, 0.0          # h1 = (0.25, 0): a2 = 1.0
    z, (Xc, a1, h1, a2, h2) = mlp.forward(theta, X)
    h7 = np.array([0.0, 8.5, 0.0, 1.0])
    assert np.array_equal(h2[:, 7], h7)
    assert np.count_nonzero(h2[:, :7]) == 0 and np.count_nonzero(h2[:, 8:]) == 0
    t = np.arange(21, dtype=float)
    assert np.array_equal(z, h7[:, None] * t[None, :] - t[None, :])
