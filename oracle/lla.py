"""Folded-concave penalties by local linear approximation (test infrastructure).

This module is test infrastructure, like the rest of oracle/: only the tests,
the smoke check and the benchmark's CPU legs may import it.

Section 6 (Extension to Non-Convex Penalty), eq. scad and eq. mcp, Algorithm 2:
the objective (1/n) sum_i rho_tau(y_i - x_i^T beta) + sum_j p_lambda(|beta_j|)
with a folded concave p_lambda is solved by the L-step local linear
approximation. Step 0 is the weighted-l1 fit with lambda_j = lambda (here
lambda omega_j, so that unpenalised columns stay unpenalised); step l
replaces the penalty by its linearisation at beta~^{l-1}, i.e. the weighted-l1
problem with lambda_j = p'_lambda(|beta~_j^{l-1}|) (times omega_j), solved by
Algorithm 1 from the previous solution (beta~, z~, theta~)^{l-1}.
"""
from __future__ import annotations

import numpy as np

from oracle import fsqrppa as O


def scad_deriv(t, lam, a=3.7):
    """eq. scad: lam for t <= lam, (a lam - t)/(a - 1) for lam < t < a lam, 0 beyond."""
    t = np.abs(np.asarray(t, dtype=np.float64))
    return np.where(t <= lam, lam, np.where(t < a * lam, (a * lam - t) / (a - 1.0), 0.0))


def mcp_deriv(t, lam, a=3.0):
    """eq. mcp: lam - t/a for t <= a lam, 0 beyond."""
    t = np.abs(np.asarray(t, dtype=np.float64))
    return np.where(t <= a * lam, lam - t / a, 0.0)


def scad_penalty(t, lam, a=3.7):
    """The SCAD penalty whose derivative is eq. scad (Fan and Li's closed form)."""
    t = np.abs(np.asarray(t, dtype=np.float64))
    mid = (2.0 * a * lam * t - t * t - lam * lam) / (2.0 * (a - 1.0))
    return np.where(t <= lam, lam * t, np.where(t < a * lam, mid, lam * lam * (a + 1.0) / 2.0))


def mcp_penalty(t, lam, a=3.0):
    """The MCP penalty whose derivative is eq. mcp (Zhang's closed form)."""
    t = np.abs(np.asarray(t, dtype=np.float64))
    return np.where(t <= a * lam, lam * t - t * t / (2.0 * a), a * lam * lam / 2.0)


DERIVS = {"scad": scad_deriv, "mcp": mcp_deriv}
PENALTIES = {"scad": scad_penalty, "mcp": mcp_penalty}


def lla_weights(beta, lam, omega, penalty, a):
    """lambda_j^l = omega_j p'_lambda(|beta_j|) for j >= 1, lambda_0 = 0 (Algorithm 2)."""
    w = omega * DERIVS[penalty](beta, lam, a)
    w[0] = 0.0
    return w


def concave_objective(Xt, y, beta, tau, lam, omega, penalty, a):
    """(1/n) sum rho_tau(y - X~ beta) + sum_{j>=1} omega_j p_lambda(|beta_j|) (omega_j in {0, 1})."""
    n = len(y)
    pen = omega[1:] * PENALTIES[penalty](beta[1:], lam, a)
    return O.pinball(y - Xt @ beta, tau).sum() / n + float(np.sum(pen))


def lla_fit(Xt, y, tau, lam, omega, block_ptr, eta, mu, penalty, a, L=1, tol=1e-6, max_iter=400000,
            check_every=10, lam_norm=1.0):
    """Algorithm 2: the weighted-l1 fit at lambda omega, then L reweighted fits,
    each started from the previous solution. Returns the list of the L + 1
    results (oracle Result objects) and the weights of each step."""
    lam_vec = lam * omega
    res = O.fsqrppa(Xt, y, tau, lam_vec, block_ptr, eta, mu, tol=tol, max_iter=max_iter,
                    check_every=check_every, lam_norm=lam_norm)
    out, weights = [res], [lam_vec]
    for _ in range(L):
        w = lla_weights(res.beta, lam, omega, penalty, a)
        res = O.fsqrppa(Xt, y, tau, w, block_ptr, eta, mu, beta0=res.beta, z0=res.z, theta0=res.theta,
                        tol=tol, max_iter=max_iter, check_every=check_every, lam_norm=lam_norm)
        out.append(res)
        weights.append(w)
    return out, weights
