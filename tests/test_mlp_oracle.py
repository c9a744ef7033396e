"""Pins of the FP64 reference of the rank-proposal network (oracle/mlp.py)
against what the mathematics fixes: central finite differences, a closed
form through a single path of units, the bfloat16 format's rounding rule
and Adam's first steps in closed form."""
import numpy as np
import pytest

from oracle import mlp
from paper_1609_08130_gb300 import inputs


def _theta(seed=3, scale=1.0):
    return mlp.init_params(inputs.uniform(seed, mlp.NPARAM)) * scale + \
        np.concatenate([np.zeros(mlp.NPARAM - 1), [0.1]])


def _data(seed=5, n=7):
    X = (inputs.uniform(seed, n * mlp.NFEAT).reshape(n, mlp.NFEAT) - 0.5) * 2.0
    X[:, 12:] = 0.0
    y = inputs.uniform(seed + 1, n)
    return X, y


def test_nparam():
    assert mlp.NPARAM == 64 * 16 + 64 + 2 * (64 * 64 + 64) + 64 + 1 == 9473


def test_backward_matches_central_differences():
    theta = _theta()
    # give the biases non-zero values so their gradients are exercised
    theta = theta + 0.05 * (inputs.uniform(11, mlp.NPARAM) - 0.5)
    X, y = _data()
    g = mlp.backward(theta, X, y)
    idx = np.unique(np.concatenate([
        (inputs.splitmix64(21, 60) % np.uint64(mlp.NPARAM)).astype(np.int64),
        [0, 1023, 1024, 1087, 1088, 5183, 5184, 5247, 5248, 9343, 9344, 9407, 9408, 9471, 9472]]))
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss(tp, X, y) - mlp.loss(tm, X, y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_forward_single_path_closed_form():
    """Only the path input 0 -> h1[1] -> h2[0] -> h3[2] -> output is non-zero,
    so o = f tanh(e tanh(c tanh(a x0))) + g0.  A transposed weight matrix or a
    layer applied out of order routes nothing to the output."""
    p = {name: np.zeros(shp) for name, shp in mlp.SHAPES}
    a, c, e, f, g0 = 0.7, -1.3, 0.9, 2.0, 0.25
    p["W1"][1, 0] = a
    p["W2"][0, 1] = c
    p["W3"][2, 0] = e
    p["w4"][2] = f
    p["b4"][0] = g0
    theta = mlp.pack(p)
    X = np.zeros((3, mlp.NFEAT))
    X[:, 0] = [-1.0, 0.3, 2.0]
    X[:, 5] = 9.0  # no weight reads it
    o, _ = mlp.forward(theta, X)
    want = f * np.tanh(e * np.tanh(c * np.tanh(a * X[:, 0]))) + g0
    np.testing.assert_allclose(o, want, rtol=0, atol=1e-15)


def test_zero_gradient_at_exact_fit():
    theta = _theta()
    X, _ = _data()
    y, _ = mlp.forward(theta, X)
    assert np.abs(mlp.backward(theta, X, y)).max() == 0.0


def test_bf16_rounding_rule():
    # bfloat16 has 8 significant bits: the spacing just above 1 is 2^-7
    cases = {
        1.0: 1.0,
        1.0 + 2.0 ** -8: 1.0,                      # halfway, ties to even (down)
        1.0 + 3 * 2.0 ** -8: 1.0 + 2.0 ** -6,      # halfway, ties to even (up)
        1.0 + 2.0 ** -8 + 2.0 ** -20: 1.0 + 2.0 ** -7,
        -(1.0 + 2.0 ** -8 + 2.0 ** -20): -(1.0 + 2.0 ** -7),
        3.14159: 3.140625,
        0.0: 0.0,
    }
    got = mlp.bf16_round(np.array(list(cases.keys()), dtype=np.float32))
    np.testing.assert_array_equal(got, np.array(list(cases.values())))


def test_adam_first_steps_closed_form():
    """With a constant gradient g the bias-corrected moments are g and g^2 at
    every step, so each step moves theta by lr g / (|g| + eps)."""
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    m = np.zeros(3)
    v = np.zeros(3)
    lr, eps = 0.01, 1e-8
    t1, m, v = mlp.adam_step(theta, m, v, g, 1, lr, eps=eps)
    np.testing.assert_allclose(t1, theta - lr * g / (np.abs(g) + eps), rtol=1e-14)
    t2, m, v = mlp.adam_step(t1, m, v, g, 2, lr, eps=eps)
    np.testing.assert_allclose(t2, t1 - lr * g / (np.abs(g) + eps), rtol=1e-12)


def test_init_params_ranges():
    u = inputs.uniform(3, mlp.NPARAM)
    p = mlp.unpack(mlp.init_params(u))
    s1 = np.sqrt(6.0 / (16 + 64))
    s2 = np.sqrt(6.0 / (64 + 64))
    s4 = np.sqrt(6.0 / (64 + 1))
    assert np.abs(p["W1"]).max() <= s1 and np.abs(p["W1"]).max() > 0.9 * s1
    assert np.abs(p["W2"]).max() <= s2 and np.abs(p["W3"]).max() <= s2
    assert np.abs(p["w4"]).max() <= s4
    for b in ("b1", "b2", "b3", "b4"):
        assert not p[b].any()
    # first weight from the first uniform number
    assert p["W1"][0, 0] == pytest.approx((2 * u[0] - 1) * s1, rel=1e-15)
