"""Edge cases of the CUDA path against the FP64 oracle, through the C ABI:
one block (G = 1), a block of one column, no feature columns (p = 0), very few
samples (n = 1, 7, 15), a constant (monomorphic) column, 2-bit storage with
covariates, and non-finite values (NaN in y is rejected before any launch;
NaN reaching the iterates through an unstandardised covariate stops the fit
with FSQR_ENUMERIC).
"""
import math

import numpy as np
import pytest

from oracle import fsqrppa as O
from oracle.lp import lp_solve
from paper_2601_02826_gb300 import synth
from tests.gpu_helpers import max_rel, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2601_02826_gb300 import fsqr
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = fsqr.Context(0, torch.cuda.current_stream().cuda_stream)
    yield c
    c.close()


def _design(ctx, w, standardize=1):
    from paper_2601_02826_gb300.device import upload
    return upload(ctx, w, standardize=standardize)


def _fit(ctx, dw, w, tau, lam_s, bp, mu, eta, n_iter, precision, tol=0.0, allowed=None):
    from paper_2601_02826_gb300 import fsqr
    beta = torch.zeros(w.P, dtype=torch.float64, device="cuda")
    z = torch.zeros(w.n, dtype=torch.float64, device="cuda")
    th = torch.zeros(w.n, dtype=torch.float64, device="cuda")
    kw = {} if allowed is None else dict(allowed=allowed)
    opts = dict(tol=tol, max_iter=n_iter, precision=precision)
    if mu is not None:
        opts.update(mu=mu, eta=eta)
    rc, info = ctx.fit(dw.design, dw.y, tau, lam_s, dw.omega, bp, beta, z, th, opts=opts, **kw)
    return rc, info, to_np(beta), to_np(z), to_np(th)


def _iterates_match(ctx, w, bp, tau=0.4, frac=0.25, n_iter=30, precisions=(0, 1), standardize=True):
    d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov, standardize=standardize)
    lmax = O.lambda_max(d.Xt, w.y, tau, w.omega)
    lam_s = frac * lmax if lmax > 0 else 0.1
    mu = O.default_mu(w.y)
    eta = O.eta_blocks(d.Xt, bp, mu)
    ref = O.fsqrppa(d.Xt, w.y, tau, lam_s * w.omega, bp, eta, mu, tol=0.0, max_iter=n_iter)
    dw = _design(ctx, w, 1 if standardize else 0)
    for prec in precisions:
        rc, info, b, z, t = _fit(ctx, dw, w, tau, lam_s, bp, mu, eta, n_iter, prec)
        tol = 1e-9 if prec == 0 else 1e-7
        assert info.iters == n_iter
        assert max_rel(b, ref.beta) <= tol, prec
        assert max_rel(z, ref.z) <= tol, prec
        assert max_rel(t, ref.theta) <= tol, prec
    return d, ref


@pytest.mark.parametrize("sizes", [[1], "one-column-block"])
def test_single_block_and_single_column_block(ctx, sizes):
    w = synth.tiny_geno(501, 290, 700, c=2, fmt=1, G=3, taus=(0.5,))
    if sizes == [1]:
        bp = np.array([0, w.P], dtype=np.int64)                      # G = 1
    else:
        bp = np.array([0, 40, 41, 300, w.P], dtype=np.int64)         # block 2 holds one column
    _iterates_match(ctx, w, bp)


@pytest.mark.parametrize("c", [0, 3])
def test_no_feature_columns(ctx, c):
    """p = 0: the intercept (and covariates) only; with c = 0 the converged
    intercept is an LP-optimal value, a sample tau-quantile."""
    from paper_2601_02826_gb300 import fsqr
    rng = np.random.default_rng(502)
    n, tau = 203, 0.3
    y = rng.standard_t(3, size=n)
    cov = rng.standard_normal((c, n))
    P = 1 + c
    omega = np.ones(P)
    omega[0] = 0.0
    w = synth.Workload("p0", n, 0, c, synth.FMT_INT8, np.zeros((0, 16), dtype=np.int8), 16, cov, y, [tau],
                       [P], omega, [0.1])
    d = O.build_design(np.zeros((0, n), dtype=np.int8), cov)
    lmax = O.lambda_max(d.Xt, y, tau, omega) if c else 0.0
    lam_s = 0.2 * lmax if c else 0.0
    mu = O.default_mu(y)
    bp = w.block_ptr()
    eta = O.eta_blocks(d.Xt, bp, mu)
    dw = _design(ctx, w)
    for prec in (0, 1):
        rc, info, b, z, t = _fit(ctx, dw, w, tau, lam_s, bp, mu, eta, 900000, prec, tol=1e-6)
        assert rc == fsqr.OK, prec
        assert O.kkt(d.Xt, y, tau, lam_s * omega, lmax if lmax > 0 else 1.0, b, z, t).value <= 1.001e-6
        _, obj_lp = lp_solve(d.Xt, y, tau, lam_s * omega)
        assert O.objective(d.Xt, y, b, tau, lam_s * omega) == pytest.approx(obj_lp, rel=1e-6)
        if c == 0:
            ys = np.sort(y)
            k = math.ceil(n * tau)
            slack = 1e-5 * (1.0 + np.max(np.abs(y)))  # the stop test's R_p scale
            assert ys[k - 1] - slack <= b[0] <= ys[min(k, n - 1)] + slack


@pytest.mark.parametrize("n", [1, 7, 15])
def test_very_few_samples(ctx, n):
    w = synth.tiny_geno(503 + n, n, 40, c=1, fmt=1, G=2, taus=(0.5,))
    _iterates_match(ctx, w, w.block_ptr())


def test_monomorphic_column_stays_zero(ctx):
    w = synth.tiny_geno(507, 260, 500, c=1, fmt=1, G=3, taus=(0.5,))
    g = w.geno.copy()
    g[[3, 77, 400], :w.n] = 1  # three constant columns (sd = 0)
    w.geno = g
    d, ref = _iterates_match(ctx, w, w.block_ptr(), n_iter=60)
    j = 1 + w.c + np.array([3, 77, 400])
    assert np.all(d.sd[j] == 0.0) and np.all(ref.beta[j] == 0.0)
    dw = _design(ctx, w)
    lmax = O.lambda_max(d.Xt, w.y, 0.4, w.omega)
    mu = O.default_mu(w.y)
    eta = O.eta_blocks(d.Xt, w.block_ptr(), mu)
    for prec in (0, 1):
        _, _, b, _, _ = _fit(ctx, dw, w, 0.4, 0.25 * lmax, w.block_ptr(), mu, eta, 60, prec)
        assert np.all(b[j] == 0.0)


def test_two_bit_storage_with_covariates(ctx):
    w = synth.tiny_geno(508, 333, 1100, c=3, fmt=2, G=4, taus=(0.5,))
    _iterates_match(ctx, w, w.block_ptr(), precisions=(0,))


def test_nan_in_y_is_rejected_before_any_launch(ctx):
    from paper_2601_02826_gb300 import fsqr
    w = synth.tiny_geno(509, 100, 60, c=0, fmt=1, G=2, taus=(0.5,))
    w.y = w.y.copy()
    w.y[17] = np.nan
    dw = _design(ctx, w)
    ctx.profile(enable=False, reset=True)
    for prec in (0, 1):
        with pytest.raises(fsqr.FsqrError) as e:
            _fit(ctx, dw, w, 0.5, 0.1, w.block_ptr(), None, None, 100, prec)
        assert e.value.code == fsqr.ENUMERIC
    # only the set-up reductions ran (column statistics, the y check): no iteration
    assert ctx.profile().iterations == 0


def test_non_finite_design_values_are_rejected(ctx):
    """A NaN or infinite covariate (or dense stored) value is reported as
    FSQR_ENUMERIC by the column statistics, before the iteration."""
    from paper_2601_02826_gb300 import fsqr
    for bad in (np.nan, np.inf):
        w = synth.tiny_geno(510, 150, 80, c=2, fmt=1, G=2, taus=(0.5,))
        w.cov = w.cov.copy()
        w.cov[1, 5] = bad
        for std in (0, 1):
            dw = _design(ctx, w, standardize=std)
            b = torch.zeros(w.P, dtype=torch.float64, device="cuda")
            z = torch.zeros(w.n, dtype=torch.float64, device="cuda")
            th = torch.zeros(w.n, dtype=torch.float64, device="cuda")
            with pytest.raises(fsqr.FsqrError) as e:
                ctx.fit(dw.design, dw.y, 0.5, 0.01, dw.omega, w.block_ptr(), b, z, th, opts=dict(precision=1))
            assert e.value.code == fsqr.ENUMERIC and "covariate" in str(e.value)


@pytest.mark.parametrize("precision", [0, 1])
def test_nan_in_the_iterate_stops_with_enumeric(ctx, precision):
    """A NaN in a given start (theta) reaches the stop test's sum of theta:
    the fit stops with FSQR_ENUMERIC at its first check instead of running on,
    and the context keeps working."""
    from paper_2601_02826_gb300 import fsqr
    w = synth.tiny_geno(512, 150, 80, c=1, fmt=1, G=2, taus=(0.5,))
    dw = _design(ctx, w)
    b = torch.zeros(w.P, dtype=torch.float64, device="cuda")
    z = torch.from_numpy(w.y.copy()).cuda()
    th = torch.zeros(w.n, dtype=torch.float64, device="cuda")
    th[7] = float("nan")
    rc, info = ctx.fit(dw.design, dw.y, 0.5, 0.05, dw.omega, w.block_ptr(), b, z, th,
                       opts=dict(tol=1e-6, max_iter=1000, precision=precision, warm=1), allowed=(fsqr.ENUMERIC,))
    assert rc == fsqr.ENUMERIC and info.status == fsqr.ENUMERIC and info.iters == 0
    dw2 = _design(ctx, synth.tiny_geno(511, 150, 80, c=2, fmt=1, G=2, taus=(0.5,)))
    assert ctx.lambda_max(dw2.design, dw2.y, 0.5, dw2.omega) > 0
