"""Shared set-up for the GPU parity tests: oracle-side design and parameters.

Everything the CUDA path is compared against comes from oracle/ here.
"""
import numpy as np

from oracle import fsqrppa as O


def oracle_problem(w, tau, frac, standardize=True, G=None):
    g = O.decode_stored(w.geno, w.fmt, w.n)
    d = O.build_design(g, w.cov, standardize=standardize)
    lmax = O.lambda_max(d.Xt, w.y, tau, w.omega)
    lam_scalar = frac * lmax
    lam = lam_scalar * w.omega
    mu = O.default_mu(w.y)
    bp = w.block_ptr()
    eta = O.eta_blocks(d.Xt, bp, mu)
    return d, lmax, lam_scalar, lam, mu, bp, eta


def to_np(t):
    return t.detach().cpu().numpy()


def max_rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / (1.0 + np.max(np.abs(b)))) if a.size else 0.0


_MEMO = {}


def memo(key, fn):
    """fn() once per key in a test session. The oracle is deterministic, so a
    converged oracle solve that several parametrised tests compare against
    (the same problem solved in another precision or slot count) runs once."""
    if key not in _MEMO:
        _MEMO[key] = fn()
    return _MEMO[key]
