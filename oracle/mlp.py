"""Oracle of the learned warm start: a plain FP64 multilayer perceptron (test infrastructure).

This module is test infrastructure, like the rest of oracle/: only the tests,
the smoke check and the benchmark's CPU legs may import it, and it shares no
code with the CUDA path.

The paper warm-starts each fit of a lambda path from the previous solution
(Section 7). The learned warm start extends that idea: a small network maps
per-feature inputs of a new (tau, lambda) to a starting coefficient. The
paper defines no such network, so this oracle states the definitions the
CUDA kernels implement:

  inputs of feature j >= 1 of a fit (tau, lambda):
      u_j = (tau, lambda / lambda_max(tau), x~_j^T v / (n lambda_max(tau))),
      v_i = tau - 1{y_i < y_(ceil(n tau))}     (the lambda_max direction);
  network: h_0 = u, h_{l+1} = relu(h_l W_l + b_l) for l < L-1,
      f = h_{L-1} W_{L-1} + b_{L-1}  (one output);
  start: beta_0 = y_(ceil(n tau)), beta_j = sd(y) f(u_j), z = y - X~ beta,
      theta_i = (tau - 1{z_i < 0}) / n  (a subgradient of the loss at z);
  training loss: sum_r w_r (f(u_r) - t_r)^2 / sum_r w_r with t_r = beta*_j / sd(y);
  optimiser: Adam (Kingma and Ba, 2015) with bias correction.

Parameter layout (flat, shared with the device kernels as an interface):
W_0 (d_0 x d_1, row-major: W[i * d_1 + o]), b_0 (d_1), W_1, b_1, ..., in order.
"""
from __future__ import annotations

import math

import numpy as np

DIMS = (3, 256, 256, 256, 1)


def param_count(dims=DIMS) -> int:
    return sum(a * b + b for a, b in zip(dims[:-1], dims[1:]))


def unpack(params, dims=DIMS):
    """Views (W_l, b_l) of the flat parameter vector."""
    out, o = [], 0
    for a, b in zip(dims[:-1], dims[1:]):
        W = params[o:o + a * b].reshape(a, b)
        o += a * b
        bias = params[o:o + b]
        o += b
        out.append((W, bias))
    assert o == len(params)
    return out


def forward(params, x, dims=DIMS):
    """Returns the output f (rows) and the list of layer outputs h_0..h_L."""
    hs = [np.asarray(x, dtype=np.float64)]
    layers = unpack(np.asarray(params, dtype=np.float64), dims)
    for l, (W, b) in enumerate(layers):
        z = hs[-1] @ W + b
        hs.append(np.maximum(z, 0.0) if l < len(layers) - 1 else z)
    return hs[-1][:, 0], hs


def loss(params, x, t, w, dims=DIMS):
    f, _ = forward(params, x, dims)
    return float(np.sum(w * (f - t) ** 2) / np.sum(w))


def grad(params, x, t, w, dims=DIMS):
    """Analytic gradient of loss() by backpropagation; returns (loss, flat gradient)."""
    f, hs = forward(params, x, dims)
    layers = unpack(np.asarray(params, dtype=np.float64), dims)
    ws = float(np.sum(w))
    g = (2.0 * w * (f - t) / ws)[:, None]           # dL/dz of the output layer
    parts = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        gW = hs[l].T @ g
        gb = g.sum(axis=0)
        parts[l] = (gW, gb)
        if l > 0:
            g = (g @ W.T) * (hs[l] > 0.0)           # through relu of layer l-1's output
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in parts])
    return float(np.sum(w * (f - t) ** 2) / ws), flat


def adam_step(params, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (params, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def features(Xt, y, tau, lam_frac, omega):
    """Inputs u_j (rows j = 1..P-1) of one fit, and lambda_max(tau)."""
    from oracle.fsqrppa import lambda_max
    n = len(y)
    lmax = lambda_max(Xt, y, tau, omega)
    q = np.sort(y)[max(0, math.ceil(n * tau) - 1)]
    v = tau - (y < q).astype(np.float64)
    s = Xt[:, 1:].T @ v
    P1 = Xt.shape[1] - 1
    u = np.empty((P1, 3))
    u[:, 0] = tau
    u[:, 1] = lam_frac
    u[:, 2] = s / (n * lmax) if lmax > 0 else 0.0
    return u, lmax


def warm_start(params, Xt, y, tau, lam_frac, omega, dims=DIMS):
    """Starting (beta, z, theta) proposed by the network."""
    n = len(y)
    u, _ = features(Xt, y, tau, lam_frac, omega)
    f, _ = forward(params, u, dims)
    beta = np.empty(Xt.shape[1])
    beta[0] = np.sort(y)[max(0, math.ceil(n * tau) - 1)]
    beta[1:] = float(np.std(y)) * f
    z = y - Xt @ beta
    theta = (tau - (z < 0).astype(np.float64)) / n
    return beta, z, theta
