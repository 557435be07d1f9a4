"""Definition layer of the oracle: penalised QR as a linear program.

Test infrastructure only (imported by tests, never by the library).

The problem of Section 1 (eq. vanilla_QR with eq. weight_l1_penalty) is the
textbook LP

    min  (1/n) sum_i (tau u_i + (1 - tau) v_i) + sum_j lam_j (b+_j + b-_j)
    s.t. X~ (b+ - b-) + u - v = y,   b+, b-, u, v >= 0,

solved by scipy's HiGHS. It is the exact minimiser FS-QRPPA converges to
(Theorem 1), and is used only on tiny inputs.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import linprog


def lp_solve(Xt, y, tau, lam, perturb=None):
    n, P = Xt.shape
    c = np.concatenate([lam, lam, np.full(n, tau / n), np.full(n, (1.0 - tau) / n)])
    if perturb is not None:
        c = c + perturb
    A = np.hstack([Xt, -Xt, np.eye(n), -np.eye(n)])
    res = linprog(c, A_eq=A, b_eq=y, bounds=(0, None), method="highs",
                  options={"primal_feasibility_tolerance": 1e-10, "dual_feasibility_tolerance": 1e-10})
    if res.status != 0:
        raise RuntimeError(f"LP failed: {res.message}")
    x = res.x
    beta = x[:P] - x[P:2 * P]
    obj = float(np.sum((tau - (y - Xt @ beta < 0)) * (y - Xt @ beta)) / n + np.sum(lam * np.abs(beta)))
    return beta, obj


def lp_unique(Xt, y, tau, lam, seed=0, eps=1e-9, tol=1e-7):
    """Solves twice, the second time with a tiny random cost perturbation.

    Returns (beta, objective, unique) where unique means both solves agree
    to tol in every coefficient (a practical uniqueness certificate).
    """
    b1, o1 = lp_solve(Xt, y, tau, lam)
    n, P = Xt.shape
    rng = np.random.default_rng(seed)
    pert = eps * rng.random(2 * P + 2 * n)
    b2, _ = lp_solve(Xt, y, tau, lam, perturb=pert)
    return b1, o1, bool(np.max(np.abs(b1 - b2)) <= tol)
