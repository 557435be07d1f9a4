"""Weighted elastic-net penalty for FS-QRPPA (test infrastructure).

This module is test infrastructure, like the rest of oracle/: only the tests,
the smoke check and the benchmark's CPU legs may import it.

Section 5 closes with a remark: the weighted-l1 penalty is the case of the
weighted elastic net whose quadratic parameters vanish, and Algorithm 1
extends to it with Proposition 1 and Theorem 1 intact (the appendix with the
details is not part of the text). Reading taken here:

    Omega(beta) = sum_j lambda_j |beta_j| + (1/2) sum_j gamma_j beta_j^2,
    gamma_j = gamma omega_j  (gamma >= 0; unpenalised columns get 0).

The beta step of eq. fsppa_update minimises, per coordinate,
    lambda_j |b| + (gamma_j/2) b^2 - s_j b + (eta_g/2) (b - beta_j^k)^2,
whose solution is the soft threshold of eq. beta_update divided by
eta_g + gamma_j instead of eta_g:
    b = [ (eta_g beta_j^k + s_j - lambda_j)_+ - (-eta_g beta_j^k - s_j - lambda_j)_+ ] / (eta_g + gamma_j).
Stationarity becomes s_j - gamma_j beta_j in lambda_j d|beta_j|, so R_b of
the stop test measures dist(s_j - gamma_j beta_j, lambda_j d|beta_j|). The z
and theta steps are those of Algorithm 1.
"""
from __future__ import annotations

import numpy as np

from oracle import fsqrppa as O


def prox_beta_enet(beta_g, s_g, lam_g, gam_g, eta_g):
    """The elastic-net beta step for one block (see the module docstring)."""
    a = eta_g * beta_g + s_g
    return (np.maximum(a - lam_g, 0.0) - np.maximum(-a - lam_g, 0.0)) / (eta_g + gam_g)


def objective(Xt, y, beta, tau, lam, gam):
    """(1/n) sum_i rho_tau(y_i - x_i^T beta) + sum_j lam_j |beta_j| + (1/2) sum_j gam_j beta_j^2."""
    return O.objective(Xt, y, beta, tau, lam) + 0.5 * float(np.sum(gam * beta * beta))


def kkt(Xt, y, tau, lam, gam, lam_norm, beta, z, theta, s=None):
    """Relative KKT residual with the elastic-net stationarity for R_b."""
    if s is None:
        s = Xt.T @ theta
    return O.kkt(Xt, y, tau, lam, lam_norm, beta, z, theta, s=s - gam * beta)


def fsqrppa_enet(Xt, y, tau, lam, gam, block_ptr, eta, mu, beta0=None, z0=None, theta0=None, tol=1e-6,
                 max_iter=100000, check_every=10, lam_norm=1.0):
    """Algorithm 1 with the elastic-net beta step, in the algorithm's order:
    block products X_g^T theta^k, the beta step per block, z by eq. z_update
    from (z^k, theta^k), theta by the extrapolated dual step."""
    n, P = Xt.shape
    G = len(block_ptr) - 1
    blocks = [slice(int(block_ptr[g]), int(block_ptr[g + 1])) for g in range(G)]
    beta = np.zeros(P) if beta0 is None else np.array(beta0, dtype=np.float64)
    z = (y - Xt @ beta) if z0 is None else np.array(z0, dtype=np.float64)
    theta = np.zeros(n) if theta0 is None else np.array(theta0, dtype=np.float64)
    sigma = mu / (G + 1)
    k = 0
    while True:
        s = np.concatenate([Xt[:, b].T @ theta for b in blocks])
        if k % check_every == 0 or k >= max_iter:
            res = kkt(Xt, y, tau, lam, gam, lam_norm, beta, z, theta, s=s)
            if res.value <= tol or k >= max_iter:
                return O.Result(beta, z, theta, k, res, res.value <= tol)
        beta_new = np.empty_like(beta)
        for g, b in enumerate(blocks):
            beta_new[b] = prox_beta_enet(beta[b], s[b], lam[b], gam[b], eta[g])
        z_new = O.prox_z(z, theta, tau, n, mu)
        xb_new = sum(Xt[:, b] @ beta_new[b] for b in blocks)
        xb_old = sum(Xt[:, b] @ beta[b] for b in blocks)
        theta = theta - sigma * (2.0 * (xb_new + z_new - y) - (xb_old + z - y))
        beta, z = beta_new, z_new
        k += 1
