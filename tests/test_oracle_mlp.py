"""Pins of the FP64 reference MLP against mathematics: central finite
differences of the loss, a hand-computed one-neuron case, SiLU's closed
form, and Adam's first step."""
import math

import numpy as np

from oracle import mlp


def test_parameter_count():
    assert mlp.N_PARAMS == 9347


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = mlp.init(1) + rng.normal(0, 0.05, mlp.N_PARAMS)
    X = rng.normal(size=(7, 12))
    T = rng.normal(size=(7, 3))
    L, g = mlp.loss_and_grad(theta, X, T)
    assert abs(L - mlp.loss(theta, X, T)) < 1e-15
    idx = np.concatenate([rng.choice(mlp.N_PARAMS, 60, replace=False),
                          [0, 767, 768, 831, 832, 9151, 9152, 9346]])   # layer edges
    h = 1e-6
    for k in idx:
        e = np.zeros(mlp.N_PARAMS)
        e[k] = h
        fd = (mlp.loss(theta + e, X, T) - mlp.loss(theta - e, X, T)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(fd)), (k, fd, g[k])


def test_silu_closed_form_and_derivative():
    z = np.linspace(-8, 8, 33)
    assert np.allclose(mlp.silu(z), z / (1 + np.exp(-z)))
    h = 1e-6
    fd = (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h)
    assert np.allclose(mlp.silu_grad(z), fd, atol=1e-8)
    assert mlp.silu(0.0) == 0.0 and abs(mlp.silu_grad(0.0) - 0.5) < 1e-15


def test_single_path_by_hand():
    # only input 0 -> hidden unit 0 of each layer -> output 0 carries weight
    layers = [(np.zeros((o, i)), np.zeros(o)) for i, o in zip(mlp.SIZES[:-1], mlp.SIZES[1:])]
    w = [0.5, -1.5, 2.0, 0.25]
    for (W, _), wk in zip(layers, w):
        W[0, 0] = wk
    layers[3][1][1] = 0.75                          # bias of output 1
    theta = mlp.flatten(layers)
    x = np.zeros((1, 12))
    x[0, 0] = 1.2
    s = lambda z: z / (1 + math.exp(-z))
    a = s(0.5 * 1.2)
    a = s(-1.5 * a)
    a = s(2.0 * a)
    y, _, _ = mlp.forward(theta, x)
    assert abs(y[0, 0] - 0.25 * a) < 1e-15 and y[0, 1] == 0.75 and y[0, 2] == 0.0


def test_adam_first_step_moves_by_lr_times_sign():
    g = np.array([0.3, -2.0, 1e-3])
    th, m, v = mlp.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=0.0)
    assert np.allclose(th, -0.01 * np.sign(g))


def test_bf16_rounding():
    assert mlp.bf16_round(1.0) == 1.0
    assert mlp.bf16_round(1.0 + 2 ** -9) == 1.0               # ties to even
    assert mlp.bf16_round(1.0 + 3 * 2 ** -9) == 1.0 + 2 ** -7
    x = np.random.default_rng(2).normal(size=1000)
    assert np.all(np.abs(mlp.bf16_round(x) - x) <= np.abs(x) * 2 ** -8)


def test_skip_connection_carries_previous_impulse():
    # all parameters zero: the output is inputs 3..5 exactly
    X = np.random.default_rng(3).normal(size=(5, 12))
    Y, _, _ = mlp.forward(np.zeros(mlp.N_PARAMS), X)
    assert np.array_equal(Y, X[:, 3:6])
    # and the gradient still matches finite differences with the skip active
    theta = mlp.init(2)
    T = np.zeros((5, 3))
    L, g = mlp.loss_and_grad(theta, X, T)
    k, h = 9344, 1e-6                                   # output bias 0
    e = np.zeros(mlp.N_PARAMS)
    e[k] = h
    fd = (mlp.loss(theta + e, X, T) - mlp.loss(theta - e, X, T)) / (2 * h)
    assert abs(fd - g[k]) < 1e-8
