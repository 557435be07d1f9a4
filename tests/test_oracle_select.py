"""Pins of the selection and interval oracle (oracle/select.py), no GPU.

Section 7 defines HBIC with C_n = log p and validation-loss selection;
Section 7.1 the [q_0.1, q_0.9] intervals where a crossing counts as a miss.
The pins: hand-computed values on a four-sample example, the LP-optimal
intercept-only fit, predictions of new samples through the back-transformed
(original-scale) coefficients, and the behaviour of the criteria on a
fitted path.
"""
import math

import numpy as np
import pytest

from oracle import fsqrppa as O
from oracle import select as S
from oracle.lp import lp_solve
from paper_2601_02826_gb300 import synth


def test_hand_computed_example():
    # y = 1, 2, 3, 4; intercept-only prediction 2.5 at tau = 0.5:
    # residuals -1.5, -0.5, 0.5, 1.5 -> rho = 0.75, 0.25, 0.25, 0.75, sum 2
    Xt = np.ones((4, 3))
    Xt[:, 1] = [1.0, -1.0, 1.0, -1.0]
    Xt[:, 2] = [0.5, 0.5, -0.5, -0.5]
    y = np.array([1.0, 2.0, 3.0, 4.0])
    beta = np.array([2.5, 0.0, 0.0])
    assert S.pinball_sum(Xt, y, beta, 0.5) == 2.0
    assert S.hbic(Xt, y, beta, 0.5, 2) == pytest.approx(math.log(2.0))
    # one active feature adds log(log 4) / 4 * log 2
    beta1 = np.array([2.5, 0.0, -1.0])  # predictions 2, 2, 3, 3: residuals -1, 0, 0, 1
    assert S.pinball_sum(Xt, y, beta1, 0.5) == 1.0
    assert S.hbic(Xt, y, beta1, 0.5, 2) == pytest.approx(0.0 + math.log(math.log(4)) / 4 * math.log(2))
    # tau = 0.9 weights the positive residuals: 0.9 * 1 + 0.1 * 1
    assert S.pinball_sum(Xt, y, beta1, 0.9) == pytest.approx(1.0)
    assert S.validation_loss(Xt, y, beta1, 0.9) == pytest.approx(0.25)


def test_interval_coverage_counts_crossings_as_misses():
    Xt = np.ones((5, 1))
    y = np.array([0.0, 1.0, 2.0, 3.0, 10.0])
    cov, width, cross = S.interval_coverage(Xt, y, np.array([0.5]), np.array([3.0]))
    assert cov == pytest.approx(3 / 5) and width == pytest.approx(2.5) and cross == 0  # 1, 2, 3 covered
    cov, width, cross = S.interval_coverage(Xt, y, np.array([3.0]), np.array([0.5]))
    assert cov == 0.0 and cross == 5 and width == pytest.approx(-2.5)


def test_intercept_only_hbic_is_the_log_of_the_optimal_loss():
    """Above lambda_max the LP optimum is the intercept at the sample
    tau-quantile, and HBIC reduces to the log of its pinball loss."""
    w = synth.tiny_geno(41, 30, 12, c=0, G=2, taus=(0.3,))
    d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
    lmax = O.lambda_max(d.Xt, w.y, 0.3, w.omega)
    b, obj = lp_solve(d.Xt, w.y, 0.3, 1.5 * lmax * w.omega)
    assert S.active_count(b) == 0
    assert S.hbic(d.Xt, w.y, b, 0.3, w.p) == pytest.approx(math.log(w.n * obj), rel=1e-12)


def test_new_samples_standardised_with_training_stats_match_original_scale_predictions():
    w = synth.tiny_geno(42, 40, 15, c=2, G=2, taus=(0.5,))
    v = synth.tiny_geno(43, 25, 15, c=2, G=2, taus=(0.5,))
    d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
    rng = np.random.default_rng(0)
    beta = rng.standard_normal(w.P)
    beta[d.sd == 0] = 0.0
    Xv = S.standardise_with(d, O.decode_stored(v.geno, v.fmt, v.n), v.cov)
    # the same predictions through the original-scale coefficients
    bo = O.back_transform(d, beta)
    raw = np.vstack([v.cov, O.decode_stored(v.geno, v.fmt, v.n).astype(np.float64)])
    assert np.allclose(Xv @ beta, bo[0] + raw.T @ bo[1:], rtol=1e-12, atol=1e-12)


def test_hbic_and_validation_loss_along_a_fitted_path():
    """Along an LP-exact path the training loss does not increase as lambda
    decreases and the active set grows; HBIC and the validation loss are
    finite and select an index of the path."""
    w = synth.tiny_geno(44, 40, 10, c=0, G=2, taus=(0.5,))
    v = synth.tiny_geno(44, 40, 10, c=0, G=2, taus=(0.5,))
    d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
    lmax = O.lambda_max(d.Xt, w.y, 0.5, w.omega)
    fr = np.geomspace(1.0, 0.05, 8)
    betas = [lp_solve(d.Xt, w.y, 0.5, f * lmax * w.omega)[0] for f in fr]
    losses = [S.pinball_sum(d.Xt, w.y, b, 0.5) for b in betas]
    assert all(l1 <= l0 + 1e-9 for l0, l1 in zip(losses, losses[1:]))
    h = [S.hbic(d.Xt, w.y, b, 0.5, w.p) for b in betas]
    assert all(np.isfinite(h)) and 0 <= S.select(h) < len(fr)
    Xv = S.standardise_with(d, O.decode_stored(v.geno, v.fmt, v.n), v.cov)
    vl = [S.validation_loss(Xv, v.y, b, 0.5) for b in betas]
    assert S.select(vl) == int(np.argmin(vl))
