"""Pins of the LLA oracle (oracle/lla.py) for SCAD and MCP (no GPU).

Section 6: eq. scad and eq. mcp give p'_lambda; Algorithm 2 solves a
weighted-l1 problem with those derivatives as weights. The pins tie the
oracle to the penalties' published closed forms (by finite differences and
at their break points), to the LP solution of the reweighted problem, to the
majorise-minimise descent property of LLA, and to the LASSO limit a -> inf.
"""
import numpy as np
import pytest

from oracle import fsqrppa as O
from oracle import lla as LLA
from oracle.lp import lp_solve
from paper_2601_02826_gb300 import synth


@pytest.mark.parametrize("penalty,a", [("scad", 3.7), ("mcp", 3.0), ("scad", 2.5), ("mcp", 1.5)])
def test_derivative_is_the_derivative_of_the_penalty(penalty, a):
    lam = 0.7
    t = np.linspace(0.013, 4.0 * a * lam, 997)
    h = 1e-6
    fd = (LLA.PENALTIES[penalty](t + h, lam, a) - LLA.PENALTIES[penalty](t - h, lam, a)) / (2 * h)
    # away from the break points the central difference is exact to O(h^2)
    brk = np.array([lam, a * lam])
    far = np.min(np.abs(t[:, None] - brk[None, :]), axis=1) > 1e-4
    assert np.max(np.abs(fd[far] - LLA.DERIVS[penalty](t[far], lam, a))) <= 1e-7


def test_break_points_and_limits():
    lam = 0.4
    for a in (3.7, 2.2):
        # SCAD: lam up to lam, continuous at lam, 0 from a lam on, linear in between
        assert LLA.scad_deriv(0.0, lam, a) == lam
        assert LLA.scad_deriv(lam, lam, a) == lam
        assert LLA.scad_deriv(lam * (1 + 1e-12), lam, a) == pytest.approx(lam, rel=1e-9)
        assert LLA.scad_deriv(a * lam, lam, a) == 0.0
        mid = 0.5 * (lam + a * lam)
        assert LLA.scad_deriv(mid, lam, a) == pytest.approx(0.5 * lam, rel=1e-12)
        assert LLA.scad_penalty(10.0, lam, a) == pytest.approx(lam * lam * (a + 1) / 2)
    for a in (3.0, 1.2):
        # MCP: lam at 0, 0 from a lam on, half-way at a lam / 2
        assert LLA.mcp_deriv(0.0, lam, a) == lam
        assert LLA.mcp_deriv(a * lam, lam, a) == pytest.approx(0.0, abs=1e-15)
        assert LLA.mcp_deriv(0.5 * a * lam, lam, a) == pytest.approx(0.5 * lam)
        assert LLA.mcp_penalty(10.0, lam, a) == pytest.approx(a * lam * lam / 2)
    # derivatives are symmetric in the sign of beta and never negative
    b = np.array([-3.0, -0.5, 0.0, 0.5, 3.0])
    for f in (LLA.scad_deriv, LLA.mcp_deriv):
        v = f(b, lam, 3.0)
        assert np.all(v >= 0) and np.allclose(v, v[::-1])


def _problem(seed, tau=0.5, frac=0.25):
    w = synth.tiny_geno(seed, 36, 14, c=1, G=3, taus=(tau,))
    d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
    lmax = O.lambda_max(d.Xt, w.y, tau, w.omega)
    mu = O.default_mu(w.y)
    eta = O.eta_blocks(d.Xt, w.block_ptr(), mu)
    return w, d, lmax, frac * lmax, mu, eta


@pytest.mark.parametrize("penalty,a", [("scad", 3.7), ("mcp", 3.0)])
def test_one_step_lla_solves_the_reweighted_lp(penalty, a):
    """Step 1 of Algorithm 2 is the weighted-l1 problem with lambda_j =
    p'_lambda(|beta~^0_j|); its fit reaches that LP's optimum."""
    w, d, lmax, lam, mu, eta = _problem(31)
    steps, weights = LLA.lla_fit(d.Xt, w.y, 0.5, lam, w.omega, w.block_ptr(), eta, mu, penalty, a, L=1,
                                 tol=1e-10, lam_norm=lmax)
    assert np.allclose(weights[1], LLA.lla_weights(steps[0].beta, lam, w.omega, penalty, a))
    assert weights[1][0] == 0.0 and np.all(weights[1][w.omega == 0] == 0.0)  # unpenalised columns stay so
    _, obj_lp = lp_solve(d.Xt, w.y, 0.5, weights[1])
    obj = O.objective(d.Xt, w.y, steps[1].beta, 0.5, weights[1])
    assert obj == pytest.approx(obj_lp, rel=1e-8, abs=1e-12)


@pytest.mark.parametrize("penalty,a", [("scad", 3.7), ("mcp", 3.0)])
def test_lla_steps_do_not_increase_the_concave_objective(penalty, a):
    """LLA is a majorise-minimise scheme: the linearised penalty majorises the
    concave one, so each step's exact solution cannot increase the
    non-convex objective (up to the solver tolerance)."""
    w, d, lmax, lam, mu, eta = _problem(32, tau=0.35)
    steps, _ = LLA.lla_fit(d.Xt, w.y, 0.35, lam, w.omega, w.block_ptr(), eta, mu, penalty, a, L=3,
                           tol=1e-10, lam_norm=lmax)
    vals = [LLA.concave_objective(d.Xt, w.y, s.beta, 0.35, lam, w.omega, penalty, a) for s in steps]
    for v0, v1 in zip(vals, vals[1:]):
        assert v1 <= v0 + 1e-8, vals


def test_large_a_gives_back_the_lasso():
    """As a -> inf both derivatives tend to lambda on any bounded set, so
    the one-step LLA fit is the LASSO fit itself."""
    w, d, lmax, lam, mu, eta = _problem(33)
    for penalty in ("scad", "mcp"):
        steps, weights = LLA.lla_fit(d.Xt, w.y, 0.5, lam, w.omega, w.block_ptr(), eta, mu, penalty, 1e12, L=1,
                                     tol=1e-10, lam_norm=lmax)
        assert np.allclose(weights[1], lam * w.omega, rtol=1e-9, atol=0)
        assert np.max(np.abs(steps[1].beta - steps[0].beta)) <= 1e-8
