"""Pins of the learned-warm-start oracle (oracle/mlp.py) against facts outside it:
finite differences, closed forms of special networks, the first Adam steps,
and the lambda_max definition the inputs are scaled by."""
import math

import numpy as np
import pytest

from oracle import fsqrppa as O
from oracle import mlp as M
from paper_2601_02826_gb300 import synth

SMALL = (3, 5, 4, 1)


def _rand(seed, dims=SMALL, scale=0.7):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, M.param_count(dims))


def test_param_count_of_the_default_network():
    # 3x256 + 256, 256x256 + 256 twice, 256x1 + 1
    assert M.param_count() == 3 * 256 + 256 + 2 * (256 * 256 + 256) + 256 + 1 == 132865


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(5)
    p = _rand(1)
    x = rng.normal(size=(17, 3))
    t = rng.normal(size=17)
    w = rng.uniform(0.5, 2.0, size=17)
    L, g = M.grad(p, x, t, w, SMALL)
    assert L == pytest.approx(M.loss(p, x, t, w, SMALL), rel=1e-14)
    h = 1e-6
    num = np.empty_like(p)
    for k in range(len(p)):
        e = np.zeros_like(p)
        e[k] = h
        num[k] = (M.loss(p + e, x, t, w, SMALL) - M.loss(p - e, x, t, w, SMALL)) / (2 * h)
    assert np.max(np.abs(num - g)) <= 1e-6 * (1.0 + np.max(np.abs(g)))


def test_forward_is_the_affine_product_when_no_unit_is_clipped():
    rng = np.random.default_rng(2)
    dims = (3, 4, 1)
    W0 = rng.uniform(0.1, 1.0, (3, 4))
    b0 = rng.uniform(0.1, 1.0, 4)
    W1 = rng.normal(size=(4, 1))
    b1 = rng.normal(size=1)
    p = np.concatenate([W0.ravel(), b0, W1.ravel(), b1])
    x = rng.uniform(0.0, 1.0, (6, 3))
    f, _ = M.forward(p, x, dims)
    np.testing.assert_allclose(f, ((x @ W0 + b0) @ W1 + b1)[:, 0], rtol=1e-14)


def test_forward_of_a_fully_clipped_network_is_the_last_bias():
    dims = (3, 4, 4, 1)
    p = np.zeros(M.param_count(dims))
    layers = M.unpack(p, dims)
    layers[0][1][:] = -5.0   # every first-layer unit is negative for |x| < 1
    layers[0][0][:] = 1.0
    layers[2][1][:] = 0.37
    x = np.random.default_rng(3).uniform(-1.0, 1.0, (5, 3))
    f, _ = M.forward(p, x, dims)
    np.testing.assert_array_equal(f, np.full(5, 0.37))


def test_adam_steps_of_a_constant_gradient_have_size_lr():
    # with a constant gradient the bias-corrected moments are g and g^2, so
    # every step moves each parameter by lr * g / (|g| + eps)
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    m = np.zeros(3)
    v = np.zeros(3)
    lr = 0.01
    for k in range(1, 6):
        p, m, v = M.adam_step(p, g, m, v, k, lr)
    np.testing.assert_allclose(p, np.array([1.0, -2.0, 0.5]) - 5 * lr * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_adam_training_reduces_the_loss_of_a_smooth_target():
    rng = np.random.default_rng(4)
    x = rng.uniform(-1, 1, (256, 3))
    t = np.sin(2 * x[:, 2]) + 0.5 * x[:, 0]
    w = np.ones(256)
    p = _rand(6, SMALL, 0.5)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    L0 = M.loss(p, x, t, w, SMALL)
    for k in range(1, 301):
        _, g = M.grad(p, x, t, w, SMALL)
        p, m, v = M.adam_step(p, g, m, v, k, 0.01)
    assert M.loss(p, x, t, w, SMALL) < 0.2 * L0


def test_features_are_scaled_by_lambda_max():
    w = synth.tiny_geno(31, 90, 40, c=0, fmt=synth.FMT_INT8, G=2)
    d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
    for tau in (0.2, 0.5, 0.85):
        u, lmax = M.features(d.Xt, w.y, tau, 0.3, w.omega)
        assert lmax == pytest.approx(O.lambda_max(d.Xt, w.y, tau, w.omega), rel=1e-15)
        assert np.all(u[:, 0] == tau) and np.all(u[:, 1] == 0.3)
        # every omega_j = 1, so the largest |u_3| is exactly 1
        assert np.max(np.abs(u[:, 2])) == pytest.approx(1.0, rel=1e-12)


def test_warm_start_of_a_zero_network_is_the_intercept_only_fit():
    w = synth.tiny_geno(32, 77, 30, c=1, fmt=synth.FMT_INT8, G=2)
    d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
    tau = 0.3
    p = np.zeros(M.param_count())
    beta, z, theta = M.warm_start(p, d.Xt, w.y, tau, 0.5, w.omega)
    q = np.sort(w.y)[math.ceil(w.n * tau) - 1]
    assert beta[0] == q and np.all(beta[1:] == 0.0)
    np.testing.assert_allclose(z, w.y - q, rtol=0, atol=1e-14)
    np.testing.assert_array_equal(theta, np.where(w.y - q < 0, tau - 1.0, tau) / w.n)
    # the intercept-only fit at beta = 0 is optimal for lambda >= lambda_max
    lmax = O.lambda_max(d.Xt, w.y, tau, w.omega)
    ref = O.fsqrppa(d.Xt, w.y, tau, 1.01 * lmax * w.omega, w.block_ptr(),
                    O.eta_blocks(d.Xt, w.block_ptr(), O.default_mu(w.y)), O.default_mu(w.y),
                    tol=1e-9, max_iter=200000, lam_norm=lmax)
    assert O.objective(d.Xt, w.y, beta, tau, 1.01 * lmax * w.omega) == pytest.approx(
        O.objective(d.Xt, w.y, ref.beta, tau, 1.01 * lmax * w.omega), rel=1e-7)
