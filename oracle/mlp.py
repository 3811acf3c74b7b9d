"""FP64 reference of the warm-start network (TEST INFRASTRUCTURE ONLY).

A fully connected network n_in -> width (x depth hidden layers, GELU) -> n_out
(linear), with the mean-squared-error loss L = sum (Y - T)^2 / (n n_out). The
paper has no such network: it starts the LM from the projected guess
(Remark rem:solver). The network is the library's learned warm start (parameters
to reduced coordinates), and this module is the reference its CUDA forward and
backward kernels are checked against. Parameters are flattened layer by layer as W_l (in x out, row-major)
then b_l (out).

Pinned by the tests: central finite differences of the loss gradient, and GELU
values (0 at 0, slope 1/2 at 0, x for large x, 0 for very negative x).
"""

from __future__ import annotations

import math

import numpy as np

_ERF = np.vectorize(math.erf)


def gelu(x):
    """GELU(x) = x Phi(x) = x (1 + erf(x / sqrt 2)) / 2."""
    return 0.5 * x * (1.0 + _ERF(x / math.sqrt(2.0)))


def gelu_grad(x):
    """d GELU / dx = Phi(x) + x phi(x)."""
    return 0.5 * (1.0 + _ERF(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def layer_sizes(n_in, width, depth, n_out):
    dims = [n_in] + [width] * depth + [n_out]
    return list(zip(dims[:-1], dims[1:]))


def n_params(n_in, width, depth, n_out):
    return sum(i * o + o for i, o in layer_sizes(n_in, width, depth, n_out))


def unpack(params, n_in, width, depth, n_out):
    out, k = [], 0
    for i, o in layer_sizes(n_in, width, depth, n_out):
        W = params[k:k + i * o].reshape(i, o)
        k += i * o
        b = params[k:k + o]
        k += o
        out.append((W, b))
    return out


def forward(params, X, n_in, width, depth, n_out):
    layers = unpack(np.asarray(params, dtype=np.float64), n_in, width, depth, n_out)
    A = np.asarray(X, dtype=np.float64)
    cache = []
    for li, (W, b) in enumerate(layers):
        Z = A @ W + b
        cache.append((A, Z))
        A = gelu(Z) if li < len(layers) - 1 else Z
    return A, cache


def loss_and_grad(params, X, T, n_in, width, depth, n_out):
    """MSE loss and its gradient with respect to the flattened parameters."""
    params = np.asarray(params, dtype=np.float64)
    Y, cache = forward(params, X, n_in, width, depth, n_out)
    T = np.asarray(T, dtype=np.float64)
    n = X.shape[0]
    loss = float(np.sum((Y - T) ** 2) / (n * n_out))
    dA = 2.0 * (Y - T) / (n * n_out)
    layers = unpack(params, n_in, width, depth, n_out)
    grads = []
    for li in range(len(layers) - 1, -1, -1):
        W, b = layers[li]
        A_in, Z = cache[li]
        dZ = dA if li == len(layers) - 1 else dA * gelu_grad(Z)
        grads.append((A_in.T @ dZ, dZ.sum(axis=0)))
        dA = dZ @ W.T
    grads.reverse()
    return loss, np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
