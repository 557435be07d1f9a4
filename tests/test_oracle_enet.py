"""Pins of the elastic-net oracle (oracle/enet.py), no GPU.

The beta step against brute-force 1-D minimisation; gamma = 0 against the
weighted-l1 oracle step by step; a converged fit against a quadratic-program
solve (scipy SLSQP) of the same penalised problem, whose solution is unique
in the penalised coordinates (the ridge term makes it strongly convex there).
"""
import math

import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import enet as EN
from oracle import fsqrppa as O
from paper_2601_02826_gb300 import synth
from tests.test_oracle_pins import golden_min


def test_enet_beta_step_matches_bruteforce():
    rng = np.random.default_rng(7)
    for _ in range(300):
        b0, s = rng.normal(0, 2, 2)
        lam, gam, eta = rng.uniform(0, 1.5), rng.uniform(0, 3), rng.uniform(0.2, 4)
        f = lambda b: lam * abs(b) + 0.5 * gam * b * b - s * b + 0.5 * eta * (b - b0) ** 2
        ref = golden_min(f, -20.0, 20.0)
        got = float(EN.prox_beta_enet(np.array([b0]), np.array([s]), np.array([lam]), np.array([gam]), eta)[0])
        assert got == pytest.approx(ref, abs=1e-7)


def test_zero_ridge_is_the_weighted_l1_iteration():
    w = synth.tiny_geno(51, 40, 20, c=1, G=3, taus=(0.4,))
    d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
    lmax = O.lambda_max(d.Xt, w.y, 0.4, w.omega)
    lam = 0.3 * lmax * w.omega
    mu = O.default_mu(w.y)
    eta = O.eta_blocks(d.Xt, w.block_ptr(), mu)
    a = EN.fsqrppa_enet(d.Xt, w.y, 0.4, lam, np.zeros(w.P), w.block_ptr(), eta, mu, tol=0.0, max_iter=150)
    b = O.fsqrppa(d.Xt, w.y, 0.4, lam, w.block_ptr(), eta, mu, tol=0.0, max_iter=150)
    assert np.array_equal(a.beta, b.beta) and np.array_equal(a.theta, b.theta)


def _qp(Xt, y, tau, lam, gam):
    """min (1/n) sum (tau u + (1 - tau) v) + lam.(b+ + b-) + 1/2 sum gam (b+ - b-)^2
    s.t. X (b+ - b-) + u - v = y, all >= 0 (the textbook split, solved by SLSQP)."""
    n, P = Xt.shape
    c = np.concatenate([lam, lam, np.full(n, tau / n), np.full(n, (1 - tau) / n)])
    A = np.hstack([Xt, -Xt, np.eye(n), -np.eye(n)])

    def f(x):
        b = x[:P] - x[P:2 * P]
        return float(c @ x + 0.5 * np.sum(gam * b * b))

    def g(x):
        b = x[:P] - x[P:2 * P]
        gb = gam * b
        return c + np.concatenate([gb, -gb, np.zeros(2 * n)])

    x0 = np.concatenate([np.zeros(2 * P), np.maximum(y, 0), np.maximum(-y, 0)])
    r = minimize(f, x0, jac=g, method="SLSQP", bounds=[(0, None)] * len(x0),
                 constraints=[{"type": "eq", "fun": lambda x: A @ x - y, "jac": lambda x: A}],
                 options={"ftol": 1e-15, "maxiter": 5000})
    assert r.success, r.message
    return r.x[:P] - r.x[P:2 * P], r.fun


@pytest.mark.parametrize("seed,tau,gfrac", [(52, 0.5, 0.5), (53, 0.3, 2.0)])
def test_converged_fit_matches_the_quadratic_program(seed, tau, gfrac):
    w = synth.tiny_geno(seed, 24, 12, c=1, G=2, taus=(tau,))
    d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
    lmax = O.lambda_max(d.Xt, w.y, tau, w.omega)
    lam = 0.2 * lmax * w.omega
    gam = gfrac * lmax * w.omega
    mu = O.default_mu(w.y)
    eta = O.eta_blocks(d.Xt, w.block_ptr(), mu)
    res = EN.fsqrppa_enet(d.Xt, w.y, tau, lam, gam, w.block_ptr(), eta, mu, tol=1e-10, max_iter=800000,
                          lam_norm=lmax)
    assert res.converged
    bq, fq = _qp(d.Xt, w.y, tau, lam, gam)
    f = EN.objective(d.Xt, w.y, res.beta, tau, lam, gam)
    assert f == pytest.approx(EN.objective(d.Xt, w.y, bq, tau, lam, gam), rel=1e-7)
    assert f <= EN.objective(d.Xt, w.y, bq, tau, lam, gam) + 1e-9
    pen = w.omega > 0
    assert np.max(np.abs(res.beta[pen] - bq[pen])) <= 1e-5
    # a larger ridge shrinks the penalised coefficients
    res2 = EN.fsqrppa_enet(d.Xt, w.y, tau, lam, 4 * gam, w.block_ptr(), eta, mu, tol=1e-10, max_iter=800000,
                           lam_norm=lmax)
    assert np.sum(res2.beta[pen] ** 2) <= np.sum(res.beta[pen] ** 2) + 1e-12
    assert math.isfinite(f)
