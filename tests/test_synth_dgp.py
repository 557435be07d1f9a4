"""The paper's simulation designs (Section 7.1 eq. dgp_simulation, Section 7.2)
as generated by synth.py, checked against their definitions (no GPU): the
AR(1) correlation 0.5^|i-j|, X_1 = Phi(X~_1) in (0, 1), and the conditional
tau-quantile q_tau(x) = x^T beta* + 0.7 X_1 Phi^{-1}(tau) that the paper
derives, by the fraction of responses below it.
"""
import numpy as np
from scipy.special import ndtri

from paper_2601_02826_gb300 import synth


def test_sparse_design_follows_the_paper():
    w = synth.paper_sparse(n=6000, p=1100, seed=5)
    X = w.geno[:, :w.n]
    assert X.shape == (1100, 6000)
    c1 = np.mean([np.corrcoef(X[j], X[j + 1])[0, 1] for j in range(1, 60)])
    c2 = np.mean([np.corrcoef(X[j], X[j + 2])[0, 1] for j in range(1, 60)])
    assert abs(c1 - 0.5) < 0.02 and abs(c2 - 0.25) < 0.02
    assert 0.0 < X[0].min() and X[0].max() < 1.0 and abs(X[0].mean() - 0.5) < 0.02
    nz = {j + 1: v for j, v in enumerate(w.beta_true) if v != 0}
    assert nz == {6: 1.0, 20: -1.0, 50: 1.0, 100: -1.0, 500: 1.0, 1000: -1.0, 1100: 1.0}
    for tau in (0.3, 0.5, 0.7):
        q = w.beta_true @ X + 0.7 * X[0] * ndtri(tau)
        assert abs(np.mean(w.y <= q) - tau) < 0.02


def test_dense_design_follows_the_paper():
    w = synth.paper_dense(n=4000, p=700, seed=6, m1=100, m2=20)
    X = w.geno[:, :w.n]
    assert np.all((X[100:120] > 0) & (X[100:120] < 1))
    assert np.count_nonzero(w.beta_true) == 100
    # the scale of the noise is a nonnegative combination of the Phi columns
    r = w.y - w.beta_true @ X
    assert abs(np.median(r)) < 0.05 and np.std(r) > 0
