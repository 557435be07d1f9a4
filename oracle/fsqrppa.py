"""FS-QRPPA oracle: a plain, slow FP64 CPU implementation (test infrastructure).

This module is test infrastructure. Only the tests, the smoke check and the
CPU-baseline leg of the benchmark may import it; the library's CUDA path never
does, and the two share no code. Everything here is written for reading
against the paper, not for speed: the standardised design matrix is formed
explicitly as a dense FP64 array and every product is a plain numpy matvec.

Problem (Section 1, eq. vanilla_QR, with the weighted-l1 penalty of
eq. weight_l1_penalty):

    min_beta (1/n) sum_i rho_tau(y_i - x_i^T beta) + sum_{j>=1} lambda_j |beta_j|,
    rho_tau(u) = (tau - 1{u < 0}) u,   lambda_0 = 0 (intercept unpenalised).

Algorithm (Section 4, eq. fsppa_update, Algorithm 1): with the column blocks
X = (X_1..X_G) of eq. decompose_x, M_g = eta_g I, eta_g > mu Lambda_max(X_g^T X_g),

    beta_g^{k+1} = eq. beta_update   (soft threshold of eta_g beta_g^k + X_g^T theta^k)
    z^{k+1}      = eq. z_update      (pinball prox at z^k + theta^k / mu)
    theta^{k+1}  = theta^k - mu/(G+1) [2 (sum_g X_g beta_g^{k+1} + z^{k+1} - y)
                                         - (sum_g X_g beta_g^k + z^k - y)]

Readings where the paper is silent (its Appendix D, E and F are not part of
the text):
  * stopping test: relative KKT residual of the saddle-point conditions of
    Proposition 1, checked every K iterations (kkt below);
  * initial point: beta^0 = 0, z^0 = y, theta^0 = 0 when none is given;
  * eta_g = (1 + margin) mu Lambda_hat_g with a power-method estimate;
  * lambda_max uses the lower order statistic y_(ceil(n tau)) as intercept;
  * standardisation: mean and population sd over non-missing entries,
    missing entries imputed by the column mean (standardised value 0).

Parity: every function is pinned by tests against closed forms, brute force,
an LP solve of the same problem (lp.py) or invariants of the iteration.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


# ----------------------------------------------------------------- the loss

def pinball(u, tau):
    """rho_tau(u) = (tau - 1{u < 0}) u  (Section 1, eq. vanilla_QR)."""
    u = np.asarray(u, dtype=np.float64)
    return (tau - (u < 0)) * u


def objective(Xt, y, beta, tau, lam):
    """(1/n) sum_i rho_tau(y_i - x_i^T beta) + sum_j lam_j |beta_j|."""
    n = len(y)
    return pinball(y - Xt @ beta, tau).sum() / n + np.sum(lam * np.abs(beta))


# -------------------------------------------------------- proximal updates

def prox_beta(beta_g, s_g, lam_g, eta_g):
    """Closed-form beta update of eq. beta_update for one block.

    beta_g^{k+1} = (1/eta_g) [ (eta_g beta_g^k + X_g^T theta^k - lambda_g)_+
                               - (-eta_g beta_g^k - X_g^T theta^k - lambda_g)_+ ]
    where s_g = X_g^T theta^k.
    """
    a = eta_g * beta_g + s_g
    return (np.maximum(a - lam_g, 0.0) - np.maximum(-a - lam_g, 0.0)) / eta_g


def prox_z(z, theta, tau, n, mu):
    """Closed-form z update of eq. z_update.

    z^{k+1} = (z^k + theta^k/mu - tau/(n mu))_+ - (-z^k - theta^k/mu - (1-tau)/(n mu))_+
    """
    v = z + theta / mu
    return np.maximum(v - tau / (n * mu), 0.0) - np.maximum(-v - (1.0 - tau) / (n * mu), 0.0)


# ------------------------------------------------------------ the design

@dataclass
class Design:
    """Standardised design X~ (n x P) as a dense FP64 matrix.

    Column 0 is the intercept (all ones, never standardised), columns
    1..c the dense covariates, columns c+1..c+p the genotype (or dense
    feature) columns. mean/sd hold the per-column centring and scale used
    (mean 0, sd 1 for the intercept); sd == 0 marks a constant column,
    whose standardised column is all zero.
    """
    Xt: np.ndarray
    mean: np.ndarray
    sd: np.ndarray
    c: int
    standardize: bool


def raw_columns(geno_cols, cov_cols):
    """Stacks covariate and genotype columns feature-major; missing = NaN.

    geno_cols: (p, n) values (int8 with -1 = missing, or float64);
    cov_cols: (c, n) float64.
    """
    g = np.asarray(geno_cols)
    if g.dtype == np.int8 or g.dtype == np.uint8:
        gf = g.astype(np.float64)
        gf[g.astype(np.int16) < 0] = np.nan
    else:
        gf = g.astype(np.float64)
    return np.vstack([np.asarray(cov_cols, dtype=np.float64).reshape(-1, gf.shape[1]), gf])


def decode_stored(stored, fmt, n):
    """Decodes the library's column storage into (p, n) feature values.

    fmt 0: dense FP64, one feature column of n doubles per row;
    fmt 1: int8, one byte per sample, -1 = missing;
    fmt 2: 2-bit, sample i in bits 2*(i%4) of byte i//4 of its column,
           codes 0/1/2 = genotype, 3 = missing.
    Returns float64 (fmt 0) or int8 with -1 for missing.
    """
    a = np.asarray(stored)
    if fmt == 0:
        return np.asarray(a, dtype=np.float64)[:, :n]
    if fmt == 1:
        return a.view(np.int8)[:, :n].copy()
    if fmt == 2:
        b = a.view(np.uint8)
        p = b.shape[0]
        out = np.empty((p, n), dtype=np.int8)
        for i in range(n):
            code = ((b[:, i // 4] >> (2 * (i % 4))) & 3).astype(np.int8)
            out[:, i] = np.where(code == 3, -1, code)
        return out
    raise ValueError(fmt)


def build_design(geno_cols, cov_cols, standardize=True):
    """Forms X~ = [1 | standardised covariates | standardised features].

    Mean imputation of missing entries (Section 7.2): a missing entry takes
    the column mean, i.e. standardised value 0.  Standardisation (Section
    7): column mean and population standard deviation over the non-missing
    entries.
    """
    F = raw_columns(geno_cols, cov_cols)           # (c + p, n), NaN = missing
    c = np.asarray(cov_cols).reshape(-1, F.shape[1]).shape[0]
    n = F.shape[1]
    miss = np.isnan(F)
    cnt = (~miss).sum(axis=1)
    Fz = np.where(miss, 0.0, F)
    mean = np.where(cnt > 0, Fz.sum(axis=1) / np.maximum(cnt, 1), 0.0)
    dev = np.where(miss, 0.0, F - mean[:, None])
    var = np.where(cnt > 0, (dev * dev).sum(axis=1) / np.maximum(cnt, 1), 0.0)
    sd = np.sqrt(var)
    if standardize:
        with np.errstate(divide="ignore", invalid="ignore"):
            cols = np.where(sd[:, None] > 0, dev / sd[:, None], 0.0)
    else:
        cols = np.where(miss, mean[:, None], F)
    Xt = np.empty((n, 1 + F.shape[0]))
    Xt[:, 0] = 1.0
    Xt[:, 1:] = cols.T
    return Design(Xt, np.concatenate([[0.0], mean]), np.concatenate([[1.0], sd]), c, standardize)


def back_transform(design: Design, beta_std):
    """Maps coefficients of X~ back to the original feature scale (Section 7).

    x~_j = (x_j - m_j)/s_j gives X~ beta = [beta_0 - sum_j m_j beta_j/s_j]
    + sum_j x_j beta_j/s_j; constant columns map to 0.
    """
    b = np.asarray(beta_std, dtype=np.float64)
    if not design.standardize:
        return b.copy()
    out = np.zeros_like(b)
    sd = design.sd[1:]
    with np.errstate(divide="ignore", invalid="ignore"):
        w = np.where(sd > 0, b[1:] / sd, 0.0)
    out[1:] = w
    out[0] = b[0] - np.sum(design.mean[1:] * w)
    return out


# -------------------------------------------------------- setup quantities

def lambda_max(Xt, y, tau, omega):
    """Smallest lambda for which beta_{1..} = 0 is optimal (up to ties).

    With beta = 0 the intercept is the sample tau-quantile q = y_(ceil(n tau))
    and the loss subgradient is v_i = tau - 1{y_i < q}; lambda_max is
    max_{j>=1, omega_j>0} |x~_j^T v| / (n omega_j).
    """
    n = len(y)
    q = np.sort(y)[max(0, math.ceil(n * tau) - 1)]
    v = tau - (y < q).astype(np.float64)
    g = np.abs(Xt.T @ v) / n
    sel = np.arange(Xt.shape[1]) >= 1
    sel &= omega > 0
    if not np.any(sel):
        return 0.0
    return float(np.max(g[sel] / omega[sel]))


def power_lambda(Xg, max_iter=100, tol=1e-6):
    """Power-method estimate of Lambda_max(X_g^T X_g) (Section 4, step metric).

    Start v = 1/sqrt(p_g); each step u = X_g v, estimate ||u||^2 (the
    Rayleigh quotient, since ||v|| = 1), v = X_g^T u / ||X_g^T u||. Stops when
    the estimate changes by at most tol relative, or after max_iter steps.
    Returns (estimate, steps).
    """
    pg = Xg.shape[1]
    v = np.full(pg, 1.0 / math.sqrt(pg))
    lam = 0.0
    for t in range(1, max_iter + 1):
        u = Xg @ v
        lam_new = float(u @ u)
        w = Xg.T @ u
        nw = math.sqrt(float(w @ w))
        if nw == 0.0:
            return 0.0, t
        v = w / nw
        if abs(lam_new - lam) <= tol * lam_new:
            return lam_new, t
        lam = lam_new
    return lam, max_iter


def eta_blocks(Xt, block_ptr, mu, margin=0.05, max_iter=100, tol=1e-6):
    """eta_g = (1 + margin) mu Lambda_hat_g (a zero block gets (1 + margin) mu)."""
    etas = []
    for g in range(len(block_ptr) - 1):
        lam_g, _ = power_lambda(Xt[:, block_ptr[g]:block_ptr[g + 1]], max_iter, tol)
        etas.append((1.0 + margin) * mu * (lam_g if lam_g > 0 else 1.0))
    return np.array(etas)


def default_mu(y):
    """mu = 1 / (n sd(y)): the z-threshold tau/(n mu) is then tau sd(y)."""
    n = len(y)
    sdy = float(np.std(y))
    return 1.0 / (n * (sdy if sdy > 0 else 1.0))


# --------------------------------------------------------- stopping test

def _dist_l1_subgrad(s, lam, b):
    """dist(s, lam * d|b|): |s - lam sign b| if b != 0, else (|s| - lam)_+."""
    return np.where(b > 0, np.abs(s - lam), np.where(b < 0, np.abs(s + lam), np.maximum(np.abs(s) - lam, 0.0)))


def _dist_pinball_subgrad(t, z, tau):
    """dist(t, d rho_tau(z)): {tau} for z>0, {tau-1} for z<0, [tau-1, tau] at 0."""
    return np.where(z > 0, np.abs(t - tau), np.where(z < 0, np.abs(t - (tau - 1.0)),
                                                     np.maximum(np.maximum(tau - 1.0 - t, t - tau), 0.0)))


@dataclass
class KKT:
    r_p: float
    r_z: float
    r_beta: float
    r_1: float

    @property
    def value(self):
        return max(self.r_p, self.r_z, self.r_beta, self.r_1)


def kkt(Xt, y, tau, lam, lam_norm, beta, z, theta, s=None):
    """Relative KKT residual of the saddle point of eq. main_lagrangian.

    Proposition 1: (beta, z, theta) is optimal iff z = y - X~ beta,
    n theta_i in d rho_tau(z_i), X~^T theta in d Omega(beta) (so the
    intercept entry is 1^T theta = 0). Residuals:
      R_p = ||y - X~ beta - z||_inf / (1 + ||y||_inf)
      R_z = max_i dist(n theta_i, d rho_tau(z_i))
      R_b = max_{j>=1} dist(s_j, lam_j d|beta_j|) / lam_norm,  s = X~^T theta
      R_1 = |1^T theta|
    lam_norm is lambda_max (1 when lambda_max is 0).
    """
    if s is None:
        s = Xt.T @ theta
    return kkt_from_products(y, tau, lam, lam_norm, beta, z, theta, Xt @ beta, s)


def kkt_from_products(y, tau, lam, lam_norm, beta, z, theta, xb, s):
    """The residuals of kkt() given the products xb = X~ beta and s = X~^T theta
    (for designs formed one block of columns at a time)."""
    n = len(y)
    r_p = float(np.max(np.abs(y - xb - z))) / (1.0 + float(np.max(np.abs(y))))
    r_z = float(np.max(_dist_pinball_subgrad(n * theta, z, tau)))
    if len(beta) > 1:
        r_b = float(np.max(_dist_l1_subgrad(s[1:], lam[1:], beta[1:]))) / lam_norm
    else:
        r_b = 0.0
    r_1 = abs(float(np.sum(theta)))
    return KKT(r_p, r_z, r_b, r_1)


def dual_point(theta, tau, n, iters=200):
    """theta_check = clip(theta - c 1, [(tau-1)/n, tau/n]) with 1^T theta_check = 0.

    c is found by bisection: the clipped sum decreases in c and changes sign
    on [min theta - tau/n, max theta - (tau-1)/n].
    """
    lo_b, hi_b = (tau - 1.0) / n, tau / n
    a = float(np.min(theta)) - hi_b
    b = float(np.max(theta)) - lo_b
    for _ in range(iters):
        c = 0.5 * (a + b)
        f = np.sum(np.clip(theta - c, lo_b, hi_b))
        if f > 0:
            a = c
        else:
            b = c
        if b - a <= 0:
            break
    c = 0.5 * (a + b)
    return np.clip(theta - c, lo_b, hi_b)


def duality_gap(Xt, y, tau, lam, beta, theta):
    """Relative duality gap (P - D)/(1 + |P| + |D|).

    Dual of eq. main_lagrangian: max y^T theta s.t. n theta_i in [tau-1, tau],
    1^T theta = 0, |x~_j^T theta| <= lam_j (j >= 1). A feasible point is
    alpha * dual_point(theta) with alpha = min(1, min_j lam_j / |x~_j^T theta_check|).
    Defined only when every lam_j > 0 for j >= 1; returns None otherwise.
    """
    n = len(y)
    if len(lam) > 1 and np.any(lam[1:] <= 0):
        return None
    P = objective(Xt, y, beta, tau, lam)
    tc = dual_point(theta, tau, n)
    sc = np.abs(Xt.T @ tc)[1:]
    with np.errstate(divide="ignore"):
        ratios = np.where(sc > 0, lam[1:] / sc, np.inf)
    alpha = min(1.0, float(np.min(ratios))) if len(ratios) else 1.0
    D = float(y @ (alpha * tc))
    return (P - D) / (1.0 + abs(P) + abs(D)), P, D


# -------------------------------------------------------------- Algorithm 1

@dataclass
class Result:
    beta: np.ndarray
    z: np.ndarray
    theta: np.ndarray
    iters: int
    kkt: KKT
    converged: bool
    history: list = field(default_factory=list)


def fsqrppa(Xt, y, tau, lam, block_ptr, eta, mu, beta0=None, z0=None, theta0=None,
            tol=1e-6, max_iter=100000, check_every=10, lam_norm=1.0, trace=False):
    """Algorithm 1 (FS-QRPPA with weighted-l1 penalty) on the dense X~.

    The loop follows the algorithm's order: every iteration takes the G block
    products X_g^T theta^k, updates each beta_g by eq. beta_update, updates z
    by eq. z_update (from z^k and theta^k), and updates theta by the third
    line of eq. fsppa_update with the aggregated sum_g X_g beta_g. Before the
    update, every check_every iterations (and at max_iter), the stopping test
    is evaluated on the current iterate w^k = (beta^k, z^k, theta^k).
    trace=True records every iterate (small problems only).
    """
    n, P = Xt.shape
    G = len(block_ptr) - 1
    blocks = [slice(int(block_ptr[g]), int(block_ptr[g + 1])) for g in range(G)]
    beta = np.zeros(P) if beta0 is None else np.array(beta0, dtype=np.float64)
    z = (y - Xt @ beta) if z0 is None else np.array(z0, dtype=np.float64)
    theta = np.zeros(n) if theta0 is None else np.array(theta0, dtype=np.float64)
    sigma = mu / (G + 1)
    hist = []
    k = 0
    while True:
        if trace:
            hist.append((beta.copy(), z.copy(), theta.copy()))
        # X_g^T theta^k for all blocks: used by the stop test and eq. beta_update
        s = np.concatenate([Xt[:, b].T @ theta for b in blocks])
        if k % check_every == 0 or k >= max_iter:
            res = kkt(Xt, y, tau, lam, lam_norm, beta, z, theta, s=s)
            if res.value <= tol or k >= max_iter:
                return Result(beta, z, theta, k, res, res.value <= tol, hist)
        # parfor g = 1..G: eq. beta_update
        beta_new = np.empty_like(beta)
        for g, b in enumerate(blocks):
            beta_new[b] = prox_beta(beta[b], s[b], lam[b], eta[g])
        # eq. z_update (uses z^k and theta^k)
        z_new = prox_z(z, theta, tau, n, mu)
        # eq. fsppa_update, theta line, with the aggregation sum_g X_g beta_g
        xb_new = sum(Xt[:, b] @ beta_new[b] for b in blocks)
        xb_old = sum(Xt[:, b] @ beta[b] for b in blocks)
        theta = theta - sigma * (2.0 * (xb_new + z_new - y) - (xb_old + z - y))
        beta, z = beta_new, z_new
        k += 1


def h_norm_sq(Xt, block_ptr, eta, mu, G, dbeta, dz, dtheta):
    """||w||_H^2 for the metric of the variable-metric PPA form of the update.

    Writing u = (beta, z), A u = X~ beta + z, D = diag(eta_g I, mu I) and
    sigma = mu/(G+1), the update satisfies 0 in T(w^{k+1}) + H (w^{k+1} - w^k)
    with T the saddle operator of eq. main_lagrangian and
    H = [[D, A^T], [A, I/sigma]], so ||w||_H^2 = u^T D u + 2 theta^T A u + ||theta||^2/sigma.
    """
    sigma = mu / (G + 1)
    eta_col = np.repeat(eta, np.diff(block_ptr))
    Au = Xt @ dbeta + dz
    return float(np.sum(eta_col * dbeta * dbeta) + mu * dz @ dz + 2.0 * dtheta @ Au + dtheta @ dtheta / sigma)


# ------------------------------------------------------------ convenience

def setup_and_fit(design: Design, y, tau, lam_frac, omega, block_ptr, mu=None, eta=None,
                  tol=1e-6, max_iter=100000, check_every=10, margin=0.05, lam=None, **kw):
    """lambda_max, lambda_j = lambda omega_j, eta_g, then Algorithm 1 from beta = 0."""
    Xt = design.Xt
    lmax = lambda_max(Xt, y, tau, omega)
    if lam is None:
        lam = lam_frac * lmax * omega
    if mu is None:
        mu = default_mu(y)
    if eta is None:
        eta = eta_blocks(Xt, block_ptr, mu, margin)
    res = fsqrppa(Xt, y, tau, lam, block_ptr, eta, mu, tol=tol, max_iter=max_iter,
                  check_every=check_every, lam_norm=lmax if lmax > 0 else 1.0, **kw)
    return res, dict(lam=lam, lam_max=lmax, mu=mu, eta=eta)
