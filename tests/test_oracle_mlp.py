"""Pins of the FP64 reference network of the warm start (oracle/mlp.py)."""

import math

import numpy as np

from oracle import mlp


def test_gelu_values():
    x = np.array([0.0, 1e-8, 10.0, -10.0, 1.0])
    g = mlp.gelu(x)
    assert g[0] == 0.0
    assert abs(g[2] - 10.0) < 1e-12 and abs(g[3]) < 1e-12
    # slope 1/2 at 0, and GELU(1) = Phi(1) = (1 + erf(1/sqrt2))/2 (the normal CDF at 1)
    assert abs(mlp.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-15
    assert abs(g[4] - 0.8413447460685429) < 1e-15
    # derivative against central differences
    xs = np.linspace(-3, 3, 13)
    h = 1e-6
    fd = (mlp.gelu(xs + h) - mlp.gelu(xs - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(xs), fd, atol=1e-9)


def test_loss_gradient_finite_differences():
    rng = np.random.default_rng(0)
    n_in, width, depth, n_out = 2, 7, 3, 5
    npar = mlp.n_params(n_in, width, depth, n_out)
    assert npar == (2 * 7 + 7) + 2 * (7 * 7 + 7) + (7 * 5 + 5)
    p = rng.normal(size=npar) * 0.5
    X = rng.normal(size=(9, n_in))
    T = rng.normal(size=(9, n_out))
    loss, g = mlp.loss_and_grad(p, X, T, n_in, width, depth, n_out)
    Y, _ = mlp.forward(p, X, n_in, width, depth, n_out)
    assert abs(loss - np.mean((Y - T) ** 2)) < 1e-14
    for j in rng.choice(npar, 25, replace=False):
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[j] += h
        pm[j] -= h
        fd = (mlp.loss_and_grad(pp, X, T, n_in, width, depth, n_out)[0] -
              mlp.loss_and_grad(pm, X, T, n_in, width, depth, n_out)[0]) / (2 * h)
        assert abs(fd - g[j]) <= 1e-7 * max(1.0, abs(g[j])), (j, fd, g[j])


def test_linear_network_is_least_squares():
    # depth 0: a single linear layer; its gradient vanishes at the least-squares solution
    rng = np.random.default_rng(1)
    X = rng.normal(size=(40, 2))
    T = rng.normal(size=(40, 3))
    Xa = np.concatenate([X, np.ones((40, 1))], axis=1)
    sol = np.linalg.lstsq(Xa, T, rcond=None)[0]
    p = np.concatenate([sol[:2].ravel(), sol[2]])
    _, g = mlp.loss_and_grad(p, X, T, 2, 0, 0, 3)
    assert np.abs(g).max() < 1e-13
