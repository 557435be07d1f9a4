"""Pins the FP64 oracle to facts outside itself (no GPU).

Each test ties an oracle function to a closed form, brute force, a library
routine (scipy HiGHS LP, numpy eigvalsh) or an invariant that the paper's
iteration must satisfy, chosen so that a dropped term, a sign error or a
wrong index in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

from oracle import fsqrppa as O
from oracle.lp import lp_solve, lp_unique
from paper_2601_02826_gb300 import synth


def golden_min(f, a, b, tol=1e-13, it=400):
    """Golden-section minimisation of a convex scalar function on [a, b]."""
    gr = (math.sqrt(5) - 1) / 2
    c, d = b - gr * (b - a), a + gr * (b - a)
    fc, fd = f(c), f(d)
    for _ in range(it):
        if b - a < tol * (1 + abs(a) + abs(b)):
            break
        if fc < fd:
            b, d, fd = d, c, fc
            c = b - gr * (b - a)
            fc = f(c)
        else:
            a, c, fc = c, d, fd
            d = a + gr * (b - a)
            fd = f(d)
    return 0.5 * (a + b)


# ------------------------------------------------------------- prox maps

def test_prox_beta_matches_bruteforce():
    """eq. beta_update is argmin lam|b| - s b + eta/2 (b - b0)^2."""
    rng = np.random.default_rng(0)
    for _ in range(300):
        b0, s = rng.normal(size=2) * rng.choice([0.01, 1, 100])
        lam = abs(rng.normal()) * rng.choice([0, 0.1, 10])
        eta = abs(rng.normal()) * rng.choice([0.01, 1, 100]) + 1e-3
        f = lambda b: lam * abs(b) - s * b + 0.5 * eta * (b - b0) ** 2
        R = abs(b0) + abs(s) / eta + 10
        ref = golden_min(f, -R, R)
        got = O.prox_beta(np.array([b0]), np.array([s]), np.array([lam]), eta)[0]
        # golden section pins the argmin to ~sqrt(eps); the value test is sharp
        assert abs(got - ref) <= 1e-6 * (1 + abs(ref)), (b0, s, lam, eta, got, ref)
        fg = f(got)
        assert fg <= f(ref) + 1e-13 * (1 + abs(fg))
        for dlt in (1e-7, 1e-5, 1e-3):
            h = dlt * (1 + abs(got))
            assert fg <= min(f(got - h), f(got + h)) + 1e-13 * (1 + abs(fg))


def test_prox_z_matches_bruteforce():
    """eq. z_update is argmin (1/n) rho_tau(z) - theta z + mu/2 (z - z0)^2."""
    rng = np.random.default_rng(1)
    for _ in range(300):
        n = int(rng.integers(1, 1000))
        tau = float(rng.uniform(0.01, 0.99))
        mu = float(abs(rng.normal()) * rng.choice([1e-3, 1, 100]) + 1e-6)
        z0 = float(rng.normal() * rng.choice([0.01, 1, 10]))
        th = float(rng.normal() / n)
        f = lambda z: O.pinball(z, tau) / n - th * z + 0.5 * mu * (z - z0) ** 2
        R = abs(z0) + abs(th) / mu + 1 / (n * mu) + 10
        ref = golden_min(f, -R, R)
        got = O.prox_z(np.array([z0]), np.array([th]), tau, n, mu)[0]
        assert abs(got - ref) <= 1e-6 * (1 + abs(ref)), (n, tau, mu, z0, th, got, ref)
        fg = f(got)
        assert fg <= f(ref) + 1e-13 * (1 + abs(fg))
        for dlt in (1e-7, 1e-5, 1e-3):
            h = dlt * (1 + abs(got))
            assert fg <= min(f(got - h), f(got + h)) + 1e-13 * (1 + abs(fg))


def test_prox_z_exact_zero_region():
    """The pinball prox returns exact zeros on its dead zone."""
    n, mu, tau = 10, 2.0, 0.3
    v = np.linspace(-(1 - tau) / (n * mu), tau / (n * mu), 11)
    out = O.prox_z(v, np.zeros_like(v), tau, n, mu)
    assert np.all(out == 0.0)


def test_pinball_definition():
    assert O.pinball(2.0, 0.3) == pytest.approx(0.6)
    assert O.pinball(-2.0, 0.3) == pytest.approx(1.4)
    assert O.pinball(0.0, 0.9) == 0.0


# --------------------------------------------------------- design helpers

def test_standardisation_and_missing_imputation():
    rng = np.random.default_rng(2)
    g = synth.binomial_genotypes(rng, 40, rng.uniform(0.05, 0.5, 7))
    g = synth.add_missing(rng, g, 0.1)
    cov = rng.normal(size=(2, 40))
    d = O.build_design(g, cov)
    Xt = d.Xt
    assert np.all(Xt[:, 0] == 1.0)
    for j in range(1, Xt.shape[1]):
        col = Xt[:, j]
        if d.sd[j] > 0:
            raw = np.concatenate([cov, g.astype(float)])[j - 1]
            obs = (g[j - 3] >= 0) if j >= 3 else np.ones(40, bool)
            assert abs(col[obs].mean()) < 1e-12
            assert abs(np.sqrt((col[obs] ** 2).mean()) - 1) < 1e-12
            assert np.all(col[~obs] == 0.0)        # imputed by the mean
            assert np.allclose(col[obs] * d.sd[j] + d.mean[j], raw[obs])


def test_back_transform_preserves_predictions():
    rng = np.random.default_rng(3)
    g = synth.binomial_genotypes(rng, 30, rng.uniform(0.05, 0.5, 9))
    g[4] = 1                                        # a constant column
    g = synth.add_missing(rng, g, 0.05)
    cov = rng.normal(size=(1, 30))
    d = O.build_design(g, cov)
    b = rng.normal(size=d.Xt.shape[1])
    bo = O.back_transform(d, b)
    raw = np.vstack([cov, np.where(g < 0, np.nan, g.astype(float))]).T
    raw = np.where(np.isnan(raw), d.mean[1:][None, :], raw)     # mean imputation
    pred_raw = bo[0] + raw @ bo[1:]
    pred_std = d.Xt @ np.where(d.sd > 0, b, 0.0)
    assert np.allclose(pred_raw, pred_std, atol=1e-10)
    assert bo[1 + 1 + 4] == 0.0                      # constant column -> 0


def test_power_method_vs_eigvalsh():
    rng = np.random.default_rng(4)
    for n, pg in [(50, 20), (30, 60), (80, 1), (5, 5)]:
        X = rng.normal(size=(n, pg))
        ref = np.linalg.eigvalsh(X.T @ X)[-1]
        est, _ = O.power_lambda(X, max_iter=5000, tol=1e-13)
        assert est <= ref * (1 + 1e-12)
        assert est == pytest.approx(ref, rel=1e-6)
    est, _ = O.power_lambda(np.zeros((10, 3)))
    assert est == 0.0


# -------------------------------------------------------- converged fits

def _tiny(seed, n=30, p=40, tau=0.5, frac=0.3, G=3, kind="dense"):
    if kind == "dense":
        w = synth.small_dense(seed=seed, n=n, p=p, G=G, tau=tau)
    else:
        w = synth.tiny_geno(seed, n, p, c=2, G=G, taus=(tau,))
    d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
    lmax = O.lambda_max(d.Xt, w.y, tau, w.omega)
    lam = frac * lmax * w.omega
    return w, d, lmax, lam


@pytest.mark.parametrize("seed,kind,tau,frac", [(10, "dense", 0.5, 0.3), (11, "dense", 0.2, 0.5),
                                               (12, "geno", 0.7, 0.3), (13, "geno", 0.5, 0.6)])
def test_converged_fit_matches_lp(seed, kind, tau, frac):
    """Theorem 1: the iteration converges to a minimiser, which the LP finds exactly."""
    w, d, lmax, lam = _tiny(seed, tau=tau, frac=frac, kind=kind)
    mu = O.default_mu(w.y)
    eta = O.eta_blocks(d.Xt, w.block_ptr(), mu)
    res = O.fsqrppa(d.Xt, w.y, tau, lam, w.block_ptr(), eta, mu, tol=1e-10, max_iter=400000, lam_norm=lmax)
    assert res.converged
    b_lp, obj_lp, unique = lp_unique(d.Xt, w.y, tau, lam)
    obj = O.objective(d.Xt, w.y, res.beta, tau, lam)
    assert obj == pytest.approx(obj_lp, rel=1e-8, abs=1e-12)
    if unique:
        assert np.max(np.abs(res.beta - b_lp)) <= 1e-6


def test_kkt_vanishes_at_lp_solution_and_not_elsewhere():
    """The stop test is zero at an exact saddle point (LP primal + LP duals)."""
    w, d, lmax, lam = _tiny(20, tau=0.4, frac=0.3)
    from scipy.optimize import linprog
    Xt, y, tau = d.Xt, w.y, 0.4
    n, P = Xt.shape
    c = np.concatenate([lam, lam, np.full(n, tau / n), np.full(n, (1 - tau) / n)])
    A = np.hstack([Xt, -Xt, np.eye(n), -np.eye(n)])
    r = linprog(c, A_eq=A, b_eq=y, bounds=(0, None), method="highs")
    beta = r.x[:P] - r.x[P:2 * P]
    beta[np.abs(beta) < 1e-12] = 0.0
    z = r.x[2 * P:2 * P + n] - r.x[2 * P + n:]
    z[np.abs(z) < 1e-12] = 0.0
    theta = r.eqlin.marginals
    k = O.kkt(Xt, y, tau, lam, lmax, beta, z, theta)
    assert k.value <= 1e-8, k
    k2 = O.kkt(Xt, y, tau, lam, lmax, beta, z, theta * 1.1)
    assert k2.value > 1e-4
    k3 = O.kkt(Xt, y, tau, lam, lmax, beta * 1.01, z, theta)
    assert k3.value > 1e-5


def test_duality_gap_weak_duality_and_zero_at_optimum():
    w, d, lmax, lam = _tiny(21, tau=0.6, frac=0.4)
    rng = np.random.default_rng(0)
    for _ in range(20):
        b = rng.normal(size=d.Xt.shape[1]) * 0.1
        th = rng.normal(size=len(w.y)) / len(w.y)
        gap, P, D = O.duality_gap(d.Xt, w.y, 0.6, lam, b, th)
        assert P >= D - 1e-12
    mu = O.default_mu(w.y)
    eta = O.eta_blocks(d.Xt, w.block_ptr(), mu)
    res = O.fsqrppa(d.Xt, w.y, 0.6, lam, w.block_ptr(), eta, mu, tol=1e-10, max_iter=400000, lam_norm=lmax)
    gap, P, D = O.duality_gap(d.Xt, w.y, 0.6, lam, res.beta, res.theta)
    assert 0 <= gap <= 1e-7


def test_lambda_max_threshold():
    """beta_{1..} = 0 is optimal just above lambda_max and not below it."""
    w, d, lmax, _ = _tiny(22, n=31, tau=0.3)
    y, Xt, tau = w.y, d.Xt, 0.3
    b_hi, _ = lp_solve(Xt, y, tau, 1.001 * lmax * w.omega)
    assert np.max(np.abs(b_hi[1:])) <= 1e-9
    q = np.sort(y)[math.ceil(len(y) * tau) - 1]
    assert b_hi[0] == pytest.approx(q, abs=1e-9)
    b_lo, _ = lp_solve(Xt, y, tau, 0.9 * lmax * w.omega)
    assert np.max(np.abs(b_lo[1:])) > 1e-6


def test_intercept_only_gives_sample_quantile():
    rng = np.random.default_rng(5)
    y = rng.standard_t(3, size=37)
    Xt = np.ones((37, 1))
    tau = 0.3                                       # n tau non-integer: unique quantile
    mu = O.default_mu(y)
    eta = O.eta_blocks(Xt, np.array([0, 1]), mu)
    res = O.fsqrppa(Xt, y, tau, np.zeros(1), np.array([0, 1]), eta, mu, tol=1e-12, max_iter=200000)
    assert res.converged
    assert res.beta[0] == pytest.approx(np.sort(y)[math.ceil(37 * tau) - 1], abs=1e-8)


def test_block_count_does_not_change_the_fixed_point():
    w, d, lmax, lam = _tiny(24, tau=0.5, frac=0.3)
    mu = O.default_mu(w.y)
    outs = []
    for G in (1, 4, 7):
        bp = np.array([0] + list(np.cumsum(synth.equal_blocks(d.Xt.shape[1], G))))
        eta = O.eta_blocks(d.Xt, bp, mu)
        res = O.fsqrppa(d.Xt, w.y, 0.5, lam, bp, eta, mu, tol=1e-9, max_iter=400000, lam_norm=lmax)
        assert res.converged
        outs.append(res.beta)
    _, _, unique = lp_unique(d.Xt, w.y, 0.5, lam)
    assert unique
    for b in outs[1:]:
        assert np.max(np.abs(b - outs[0])) <= 1e-6


def test_reflection_symmetry():
    """rho_tau(-u) = rho_{1-tau}(u): (y, tau) -> (-y, 1 - tau) maps beta -> -beta."""
    w, d, lmax, lam = _tiny(24, tau=0.3, frac=0.3)
    mu = O.default_mu(w.y)
    eta = O.eta_blocks(d.Xt, w.block_ptr(), mu)
    r1 = O.fsqrppa(d.Xt, w.y, 0.3, lam, w.block_ptr(), eta, mu, tol=1e-10, max_iter=400000, lam_norm=lmax)
    r2 = O.fsqrppa(d.Xt, -w.y, 0.7, lam, w.block_ptr(), eta, mu, tol=1e-10, max_iter=400000, lam_norm=lmax)
    assert r1.converged and r2.converged
    assert np.max(np.abs(r1.beta + r2.beta)) <= 1e-6


def test_scale_equivariance_per_iterate():
    """y -> a y with mu -> mu/a scales every beta, z iterate by a and keeps theta."""
    w, d, lmax, lam = _tiny(25, tau=0.6, frac=0.3)
    mu = O.default_mu(w.y)
    a = 3.5
    eta = O.eta_blocks(d.Xt, w.block_ptr(), mu)
    r1 = O.fsqrppa(d.Xt, w.y, 0.6, lam, w.block_ptr(), eta, mu, tol=0, max_iter=300)
    r2 = O.fsqrppa(d.Xt, a * w.y, 0.6, lam, w.block_ptr(), eta / a, mu / a, tol=0, max_iter=300)
    assert np.allclose(r2.beta, a * r1.beta, rtol=1e-9, atol=1e-12)
    assert np.allclose(r2.z, a * r1.z, rtol=1e-9, atol=1e-12)
    assert np.allclose(r2.theta, r1.theta, rtol=1e-9, atol=1e-15)


def test_column_permutation_equivariance():
    w, d, lmax, lam = _tiny(26, tau=0.5, frac=0.3)
    rng = np.random.default_rng(7)
    P = d.Xt.shape[1]
    perm = np.concatenate([[0], 1 + rng.permutation(P - 1)])
    mu = O.default_mu(w.y)
    bp = w.block_ptr()
    eta = O.eta_blocks(d.Xt, bp, mu)
    eta_p = O.eta_blocks(d.Xt[:, perm], bp, mu)
    r1 = O.fsqrppa(d.Xt, w.y, 0.5, lam, bp, eta, mu, tol=1e-10, max_iter=400000, lam_norm=lmax)
    r2 = O.fsqrppa(d.Xt[:, perm], w.y, 0.5, lam[perm], bp, eta_p, mu, tol=1e-10, max_iter=400000, lam_norm=lmax)
    assert np.max(np.abs(r2.beta - r1.beta[perm])) <= 1e-6


# ----------------------------------------------- convergence behaviour

def _trace(seed=30, iters=600, tau=0.5, frac=0.3):
    w, d, lmax, lam = _tiny(seed, tau=tau, frac=frac)
    mu = O.default_mu(w.y)
    bp = w.block_ptr()
    eta = O.eta_blocks(d.Xt, bp, mu)
    res = O.fsqrppa(d.Xt, w.y, tau, lam, bp, eta, mu, tol=0, max_iter=iters, trace=True)
    return w, d, bp, eta, mu, lam, lmax, res


def test_successive_differences_nonincreasing_in_H():
    """PPA in the metric H: ||w^{k+2} - w^{k+1}||_H <= ||w^{k+1} - w^k||_H."""
    w, d, bp, eta, mu, lam, lmax, res = _trace()
    G = len(bp) - 1
    h = res.history
    dn = [O.h_norm_sq(d.Xt, bp, eta, mu, G, h[k + 1][0] - h[k][0], h[k + 1][1] - h[k][1], h[k + 1][2] - h[k][2])
          for k in range(len(h) - 1)]
    assert min(dn) >= -1e-14 * max(dn)              # H is positive semidefinite
    for k in range(len(dn) - 1):
        assert dn[k + 1] <= dn[k] * (1 + 1e-9) + 1e-28, k


def test_fejer_monotone_towards_solution():
    """||w^{k+1} - w_bar||_H <= ||w^k - w_bar||_H for the limit point w_bar."""
    w, d, bp, eta, mu, lam, lmax, res = _trace(iters=400)
    G = len(bp) - 1
    fin = O.fsqrppa(d.Xt, w.y, 0.5, lam, bp, eta, mu, tol=1e-13, max_iter=2_000_000, lam_norm=lmax)
    assert fin.converged
    dist = [O.h_norm_sq(d.Xt, bp, eta, mu, G, b - fin.beta, z - fin.z, t - fin.theta) for b, z, t in res.history]
    for k in range(len(dist) - 1):
        assert dist[k + 1] <= dist[k] * (1 + 1e-7) + 1e-22, k


def test_r_linear_rate():
    """Corollary 1: the error decays geometrically; Theorem 1: the KKT goes to 0."""
    w, d, lmax, lam = _tiny(31, tau=0.5, frac=0.4)
    mu = O.default_mu(w.y)
    bp = w.block_ptr()
    eta = O.eta_blocks(d.Xt, bp, mu)
    fin = O.fsqrppa(d.Xt, w.y, 0.5, lam, bp, eta, mu, tol=1e-13, max_iter=2_000_000, lam_norm=lmax)
    K = fin.iters
    res = O.fsqrppa(d.Xt, w.y, 0.5, lam, bp, eta, mu, tol=0, max_iter=int(0.8 * K), trace=True)
    err = np.array([math.sqrt(np.sum((b - fin.beta) ** 2) + np.sum((z - fin.z) ** 2) + np.sum((t - fin.theta) ** 2))
                    for b, z, t in res.history])
    ks = np.arange(len(err))
    tail = ks >= len(err) // 2
    slope = np.polyfit(ks[tail], np.log(err[tail]), 1)[0]
    assert slope < 0
    rho = math.exp(slope)
    # dist(w^k, S) <= C rho^k with the fitted rate and a constant from the tail
    C = np.max(err[tail] / rho ** ks[tail])
    assert np.all(err[tail] <= C * rho ** ks[tail] * (1 + 1e-12))
    assert err[-1] < 1e-3 * err[0]


# ---------------------------------------------------- planted mistakes

def test_planted_sign_error_in_z_prox_is_caught(monkeypatch):
    """Swapping tau and 1-tau in eq. z_update moves the fixed point off the LP optimum."""
    w, d, lmax, lam = _tiny(40, tau=0.25, frac=0.3)
    good = O.prox_z
    monkeypatch.setattr(O, "prox_z", lambda z, th, tau, n, mu: good(z, th, 1 - tau, n, mu))
    mu = O.default_mu(w.y)
    eta = O.eta_blocks(d.Xt, w.block_ptr(), mu)
    res = O.fsqrppa(d.Xt, w.y, 0.25, lam, w.block_ptr(), eta, mu, tol=1e-9, max_iter=20000, lam_norm=lmax)
    _, obj_lp = lp_solve(d.Xt, w.y, 0.25, lam)
    obj = O.objective(d.Xt, w.y, res.beta, 0.25, lam)
    assert (not res.converged) or obj > obj_lp * (1 + 1e-4)


def test_planted_threshold_error_in_beta_prox_is_caught(monkeypatch):
    """Dropping the 1/eta_g on the threshold breaks the match with the LP."""
    w, d, lmax, lam = _tiny(41, tau=0.5, frac=0.3)
    monkeypatch.setattr(O, "prox_beta", lambda b, s, l, e: np.sign(b + s / e) * np.maximum(np.abs(b + s / e) - l, 0.0))
    mu = O.default_mu(w.y)
    eta = O.eta_blocks(d.Xt, w.block_ptr(), mu)
    res = O.fsqrppa(d.Xt, w.y, 0.5, lam, w.block_ptr(), eta, mu, tol=1e-9, max_iter=20000, lam_norm=lmax)
    _, obj_lp = lp_solve(d.Xt, w.y, 0.5, lam)
    obj = O.objective(d.Xt, w.y, res.beta, 0.5, lam)
    assert (not res.converged) or obj > obj_lp * (1 + 1e-4)


# ------------------------------------------------------ genotype codec

def test_oracle_decoder_matches_generator_layout():
    rng = np.random.default_rng(18)
    g = synth.add_missing(rng, synth.binomial_genotypes(rng, 45, rng.uniform(0.05, 0.5, 6)), 0.1)
    assert np.array_equal(O.decode_stored(synth.pack_2bit(g)[0], 2, 45), g)
    assert np.array_equal(O.decode_stored(synth.store_int8(g)[0], 1, 45), g)


def test_2bit_roundtrip_and_layout():
    rng = np.random.default_rng(8)
    g = synth.binomial_genotypes(rng, 37, rng.uniform(0.05, 0.5, 5))
    g = synth.add_missing(rng, g, 0.1)
    packed, ld = synth.pack_2bit(g)
    assert ld % 16 == 0 and ld >= (37 + 3) // 4
    assert np.array_equal(synth.unpack_2bit(packed, 37), g)
    # sample i lives in bits 2*(i%4) of byte i//4
    for j in range(5):
        for i in range(37):
            code = (int(packed[j, i // 4]) >> (2 * (i % 4))) & 3
            assert code == (3 if g[j, i] < 0 else g[j, i])


def test_int8_storage_padding():
    rng = np.random.default_rng(9)
    g = synth.binomial_genotypes(rng, 21, rng.uniform(0.05, 0.5, 3))
    st, ld = synth.store_int8(g)
    assert ld == 32 and np.all(st[:, 21:] == 0)
    assert np.array_equal(synth.unpack_int8(st, 21), g)


def test_generator_is_seeded_and_stable():
    a = synth.tiny_geno(123, 50, 20)
    b = synth.tiny_geno(123, 50, 20)
    assert np.array_equal(a.geno, b.geno) and np.array_equal(a.y, b.y)
    g = synth.unpack_int8(a.geno, 50)
    assert set(np.unique(g)) <= {0, 1, 2}
    import hashlib
    h = hashlib.sha256(a.geno.tobytes()).hexdigest()[:16]
    with open(__file__.replace("test_oracle_pins.py", "golden/tiny_geno_123_50x20.sha256")) as f:
        assert f.read().split()[0] == h


def test_block_layouts():
    assert synth.equal_blocks(2001, 4) == [501, 500, 500, 500]
    rng = np.random.default_rng(0)
    bs = synth.ragged_blocks(rng, 100_000, 5000, 30000)
    assert sum(bs) == 100_000 and all(b >= 1 for b in bs) and all(b <= 30000 for b in bs)


def test_step_metric_makes_the_ppa_metric_positive_semidefinite():
    """Reading of the step condition (Section 4): with eta_g = (1 + margin) mu
    Lambda_max(X_g^T X_g) and sigma = mu/(G+1), D - sigma A^T A is positive
    semidefinite for A = [X_1 .. X_G  I] and D = diag(eta_g I, mu I), which
    makes the PPA metric H PSD. Below sigma Lambda_max it is not."""
    w = synth.tiny_geno(33, 40, 30, c=0, fmt=synth.FMT_INT8, G=3)
    d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
    Xt, bp = d.Xt, w.block_ptr()
    G = len(bp) - 1
    mu = O.default_mu(w.y)
    sigma = mu / (G + 1)
    A = np.hstack([Xt, np.eye(w.n)])

    def min_eig(eta):
        Dg = np.concatenate([np.repeat(eta, np.diff(bp)), np.full(w.n, mu)])
        return np.linalg.eigvalsh(np.diag(Dg) - sigma * A.T @ A).min()

    eta = O.eta_blocks(Xt, bp, mu, 0.05, 1000, 1e-14)
    lam = np.array([np.linalg.eigvalsh(Xt[:, bp[g]:bp[g + 1]].T @ Xt[:, bp[g]:bp[g + 1]]).max()
                    for g in range(G)])
    assert np.allclose(eta, 1.05 * mu * lam, rtol=1e-9)
    assert min_eig(eta) >= -1e-12 * np.max(eta)
    assert min_eig(mu * lam) >= -1e-12 * np.max(eta)   # the bound itself, with no margin
    assert min_eig(0.5 * sigma * lam) < 0.0
