"""Pins of the rank-bracket network oracle (CPU): central finite differences of the loss, and
closed forms of the forward pass and the loss gradient."""
import numpy as np

from oracle import mlp


def random_params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.normal(0, scale, mlp.N_PARAMS)


def test_param_count():
    assert mlp.N_PARAMS == 41 * 64 + 64 + 64 * 64 + 64 + 64 * 2 + 2 == 6978


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = random_params(2, scale=0.08)
    x = rng.normal(0, 1, (16, 41))
    y = rng.uniform(0, 1, 16)
    o, _ = mlp.forward(p, x)
    assert np.all(np.abs(o[:, 1]) < 1.5)  # away from the clamp on s: the loss is smooth here
    _, g = mlp.loss_and_grad(p, x, y)
    idx = rng.choice(mlp.N_PARAMS, 120, replace=False)
    idx = np.concatenate([idx, np.arange(mlp.N_PARAMS - 130, mlp.N_PARAMS)])  # all of W3, b3, part of b2
    eps = 1e-6
    for i in idx:
        d = np.zeros_like(p)
        d[i] = eps
        fd = (mlp.loss_only(p + d, x, y) - mlp.loss_only(p - d, x, y)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_forward_closed_forms():
    # all weights zero: o = b3 for every input
    p = np.zeros(mlp.N_PARAMS)
    w = mlp.unpack(p)
    w["b3"][:] = [0.25, -1.0]
    o, _ = mlp.forward(p, np.ones((3, 41)))
    assert np.allclose(o, [[0.25, -1.0]] * 3)
    # a single path: x0 -> hidden 0 -> hidden 0 -> mu, all weights 1: mu = relu(relu(x0))
    p = np.zeros(mlp.N_PARAMS)
    w = mlp.unpack(p)
    w["W1"][0, 0] = 1.0
    w["W2"][0, 0] = 1.0
    w["W3"][0, 0] = 1.0
    x = np.zeros((2, 41))
    x[:, 0] = [2.5, -1.0]
    o, _ = mlp.forward(p, x)
    assert np.allclose(o[:, 0], [2.5, 0.0]) and np.allclose(o[:, 1], 0.0)


def test_loss_gradient_closed_form():
    # with only b3 nonzero, dL/db3 = mean(-(y - mu) e^{-2s}), mean(1 - (y - mu)^2 e^{-2s})
    p = np.zeros(mlp.N_PARAMS)
    w = mlp.unpack(p)
    w["b3"][:] = [0.4, -0.5]
    y = np.array([0.1, 0.9, 0.4])
    loss, g = mlp.loss_and_grad(p, np.zeros((3, 41)), y)
    e = y - 0.4
    inv = np.exp(1.0)
    assert np.isclose(loss, np.mean(0.5 * e * e * inv - 0.5))
    assert np.isclose(g[-2], np.mean(-e * inv)) and np.isclose(g[-1], np.mean(1 - e * e * inv))
    assert np.allclose(g[:-2], 0.0)
    # the clamp on s stops the scale gradient outside [-8, 2]
    w["b3"][1] = 5.0
    _, g = mlp.loss_and_grad(p, np.zeros((3, 41)), y)
    assert g[-1] == 0.0


def test_bf16_values():
    bits = np.array([0x3f80, 0xbf80, 0x4049, 0x0000, 0x8000, 0x7f7f], np.uint16)
    v = mlp.bf16_values(bits)
    assert v[0] == 1.0 and v[1] == -1.0 and v[3] == 0.0 and np.signbit(v[4])
    assert abs(v[2] - 3.140625) < 1e-12
