"""Parity at the benchmark's full size: n = 5,000, p = 100,000 int8 genotypes,
5 covariates, G = 32, three quantiles advanced together on the tensor cores,
the launch configuration bench.py times.

The oracle runs Algorithm 1 on the dense standardised design (4 GB in FP64)
for a few iterations, and evaluates the stop test of the GPU's converged
output. Tolerances:
  * iterates after 20 steps from the same start: 1e-7 relative (FP64 GPU
    path: 1e-9). The mixed path rounds theta to 2^-28 of its scale each step;
    the oracle run with that rounding applied moves by at most 3e-9 (z),
    8e-11 (beta) and 6e-13 (theta) from the exact one after 20 steps;
  * converged fit: the oracle's KKT of the returned iterate <= tol.
"""
import numpy as np
import pytest

from oracle import fsqrppa as O
from paper_2601_02826_gb300 import synth
from tests.gpu_helpers import max_rel, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_2601_02826_gb300 import fsqr
    from paper_2601_02826_gb300.device import upload
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    ctx = fsqr.Context(0, torch.cuda.current_stream().cuda_stream)
    w = synth.geno_int8()
    dw = upload(ctx, w)
    d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
    yield ctx, w, dw, d
    ctx.close()


def _lams(d, w, taus, frac):
    lmax = [O.lambda_max(d.Xt, w.y, t, w.omega) for t in taus]
    return lmax, np.array([[frac * lm] for lm in lmax])


@pytest.mark.parametrize("precision,tol", [(1, 1e-7), (0, 1e-9)])
def test_full_size_iterates_match_oracle(setup, precision, tol):
    ctx, w, dw, d = setup
    taus = [0.1, 0.5, 0.9]
    lmax, lams = _lams(d, w, taus, 0.1)
    mu = O.default_mu(w.y)
    bp = w.block_ptr()
    eta = O.eta_blocks(d.Xt, bp, mu)
    B, n_it = 3, 20
    beta = torch.zeros(B * w.P, dtype=torch.float64, device="cuda")
    z = torch.zeros(B * w.n, dtype=torch.float64, device="cuda")
    th = torch.zeros(B * w.n, dtype=torch.float64, device="cuda")
    ctx.fit_batch(dw.design, dw.y, taus, lams, dw.omega, bp, beta, z, th,
                  opts=dict(tol=0.0, max_iter=n_it, mu=mu, eta=eta, precision=precision, digits=4, max_group=3))
    bb, zz, tt = to_np(beta).reshape(B, -1), to_np(z).reshape(B, -1), to_np(th).reshape(B, -1)
    for f, tau in enumerate(taus):
        ref = O.fsqrppa(d.Xt, w.y, tau, lams[f, 0] * w.omega, bp, eta, mu, tol=0.0, max_iter=n_it)
        assert max_rel(bb[f], ref.beta) <= tol, (f, max_rel(bb[f], ref.beta))
        assert max_rel(zz[f], ref.z) <= tol
        assert max_rel(tt[f], ref.theta) <= tol


def test_full_size_converged_fit_meets_the_oracle_stop_test(setup):
    """The tau = 0.5 fit of the benchmark (about 183,000 iterations)."""
    ctx, w, dw, d = setup
    tau = 0.5
    lmax, lams = _lams(d, w, [tau], 0.1)
    beta = torch.zeros(w.P, dtype=torch.float64, device="cuda")
    z = torch.zeros(w.n, dtype=torch.float64, device="cuda")
    th = torch.zeros(w.n, dtype=torch.float64, device="cuda")
    rc, info = ctx.fit(dw.design, dw.y, tau, lams[0, 0], dw.omega, w.block_ptr(), beta, z, th,
                       opts=dict(tol=1e-6, max_iter=1_000_000, precision=1, digits=4))
    assert rc == 0 and info.kkt <= 1e-6
    lam = lams[0, 0] * w.omega
    k = O.kkt(d.Xt, w.y, tau, lam, lmax[0], to_np(beta), to_np(z), to_np(th))
    assert k.value <= 1e-6 * (1 + 1e-3), k
    # the certified test is an upper bound of the FP64 one
    assert k.value <= info.kkt * (1 + 1e-9)
