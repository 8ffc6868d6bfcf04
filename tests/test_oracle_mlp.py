"""Pins of the selector's reference network (oracle.mlp): back-propagation against central
finite differences of the loss, and the Adam update on a quadratic."""

import numpy as np


def test_mlp_gradient_is_the_finite_difference_of_the_loss():
    from oracle import mlp

    rng = np.random.default_rng(9)
    n_in, n_h, n_out, B = 5, 7, 3, 11
    theta = rng.normal(scale=0.4, size=mlp.n_params(n_in, n_h, n_out))
    x = rng.normal(size=(B, n_in))
    t = rng.normal(size=(B, n_out))
    L, g = mlp.loss_and_grad(theta, x, t, n_in, n_h, n_out)
    assert abs(L - mlp.loss(theta, x, t, n_in, n_h, n_out)) < 1e-15
    h = 1e-6
    fd = np.empty_like(theta)
    for k in range(theta.size):
        e = np.zeros_like(theta)
        e[k] = h
        fd[k] = (mlp.loss(theta + e, x, t, n_in, n_h, n_out) - mlp.loss(theta - e, x, t, n_in, n_h, n_out)) / (2 * h)
    assert np.max(np.abs(fd - g)) < 1e-8 * max(1.0, np.max(np.abs(g)))


def test_mlp_adam_decreases_a_quadratic():
    from oracle import mlp

    theta, m, v = np.array([3.0, -2.0]), np.zeros(2), np.zeros(2)
    for s in range(1, 2001):
        theta, m, v = mlp.adam_step(theta, m, v, 2.0 * theta, s, 0.05)
    assert np.max(np.abs(theta)) < 1e-3
