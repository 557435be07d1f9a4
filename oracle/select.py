"""Model selection and prediction intervals along a penalty path (test infrastructure).

This module is test infrastructure, like the rest of oracle/: only the tests,
the smoke check and the benchmark's CPU legs may import it.

Section 7 (Numerical Studies), HBIC definition: in sparse settings lambda is
chosen by the high-dimensional BIC of quantile regression,
    HBIC(lambda) = log( sum_i rho_tau(y_i - x_i^T beta) ) + |A| (log log n / n) C_n,
with A the active set and C_n = log p (p candidate features); in dense
settings by the pinball loss on a validation set. Section 7.1: the
prediction interval of x is [q_0.1(x), q_0.9(x)] from the fits at tau = 0.1
and 0.9, and an interval whose ends cross counts as a miss.
"""
from __future__ import annotations

import math

import numpy as np

from oracle import fsqrppa as O


def pinball_sum(Xt, y, beta, tau):
    """sum_i rho_tau(y_i - x~_i^T beta)."""
    return float(np.sum(O.pinball(y - Xt @ beta, tau)))


def active_count(beta):
    """|A| = #{j >= 1 : beta_j != 0} (the intercept is not a selected feature)."""
    return int(np.count_nonzero(np.asarray(beta)[1:]))


def hbic(Xt, y, beta, tau, p_features):
    """HBIC(lambda) with C_n = log p."""
    n = len(y)
    return math.log(pinball_sum(Xt, y, beta, tau)) + active_count(beta) * math.log(math.log(n)) / n * math.log(
        p_features)


def validation_loss(Xt_val, y_val, beta, tau):
    """(1/n_val) sum_i rho_tau(y_i - x~_i^T beta) on held-out data (standardised
    with the training columns' mean and sd)."""
    return pinball_sum(Xt_val, y_val, beta, tau) / len(y_val)


def select(values):
    """Index of the smallest criterion value along the path (first on ties)."""
    return int(np.argmin(np.asarray(values)))


def interval_coverage(Xt, y, beta_lo, beta_hi):
    """Coverage of [q_lo, q_hi] = [x~^T beta_lo, x~^T beta_hi]: the fraction of
    samples with q_lo <= y <= q_hi where the ends do not cross; also the mean
    width q_hi - q_lo and the number of crossings q_lo > q_hi."""
    lo, hi = Xt @ beta_lo, Xt @ beta_hi
    ok = (lo <= hi) & (lo <= y) & (y <= hi)
    return float(np.mean(ok)), float(np.mean(hi - lo)), int(np.count_nonzero(lo > hi))


def standardise_with(design_train: O.Design, geno_cols, cov_cols):
    """X~ of new samples standardised with the training columns' mean and sd
    (missing entries take the training mean, i.e. 0)."""
    F = O.raw_columns(geno_cols, cov_cols)
    mean, sd = design_train.mean[1:], design_train.sd[1:]
    Fz = np.where(np.isnan(F), mean[:, None], F)
    with np.errstate(divide="ignore", invalid="ignore"):
        cols = np.where(sd[:, None] > 0, (Fz - mean[:, None]) / sd[:, None], 0.0)
    Xt = np.empty((F.shape[1], 1 + F.shape[0]))
    Xt[:, 0] = 1.0
    Xt[:, 1:] = cols.T
    return Xt
