"""Reference multilayer perceptron for the parameter selector (test infrastructure).

Part of the FP64 CPU oracle; only tests, the smoke check and the benchmark's CPU legs may
import it.  The network the selector trains on the GPU, written out plainly:

    a1 = W1 x + b1,  h1 = tanh(a1)
    a2 = W2 h1 + b2, h2 = tanh(a2)
    y  = W3 h2 + b3
    L  = (1 / (B n_out)) sum_b sum_o (y_bo - t_bo)^2

Parameters are one flat vector in the order W1 (n_h x n_in, row-major), b1, W2 (n_h x n_h),
b2, W3 (n_out x n_h), b3.  ``loss_and_grad`` is back-propagation by the chain rule; the
tests pin it to central finite differences of ``loss``.
"""

from __future__ import annotations

import numpy as np


def shapes(n_in: int, n_h: int, n_out: int):
    return [(n_h, n_in), (n_h,), (n_h, n_h), (n_h,), (n_out, n_h), (n_out,)]


def unpack(theta, n_in, n_h, n_out):
    out, k = [], 0
    for s in shapes(n_in, n_h, n_out):
        size = int(np.prod(s))
        out.append(np.asarray(theta[k:k + size], dtype=np.float64).reshape(s))
        k += size
    return out


def n_params(n_in, n_h, n_out):
    return sum(int(np.prod(s)) for s in shapes(n_in, n_h, n_out))


def forward(theta, x, n_in, n_h, n_out):
    W1, b1, W2, b2, W3, b3 = unpack(theta, n_in, n_h, n_out)
    x = np.asarray(x, dtype=np.float64)
    h1 = np.tanh(x @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h2 @ W3.T + b3, (x, h1, h2)


def loss(theta, x, t, n_in, n_h, n_out):
    y, _ = forward(theta, x, n_in, n_h, n_out)
    t = np.asarray(t, dtype=np.float64)
    return float(np.mean((y - t) ** 2))


def loss_and_grad(theta, x, t, n_in, n_h, n_out):
    W1, b1, W2, b2, W3, b3 = unpack(theta, n_in, n_h, n_out)
    y, (x, h1, h2) = forward(theta, x, n_in, n_h, n_out)
    t = np.asarray(t, dtype=np.float64)
    B = x.shape[0]
    d3 = 2.0 * (y - t) / (B * n_out)          # dL/dy
    gW3 = d3.T @ h2
    gb3 = d3.sum(axis=0)
    d2 = (d3 @ W3) * (1.0 - h2 * h2)          # dL/da2
    gW2 = d2.T @ h1
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * (1.0 - h1 * h1)          # dL/da1
    gW1 = d1.T @ x
    gb1 = d1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return float(np.mean((y - t) ** 2)), g


def adam_step(theta, m, v, g, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015) with bias correction; returns new arrays."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
