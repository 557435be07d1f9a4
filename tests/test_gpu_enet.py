"""Weighted elastic net (opts.ridge, Section 5 closing remark) on the GPU
against oracle/enet.py, through the C ABI: iterates after N steps on every
path (FP64 SIMT, tensor-core groups, wide slots) and converged fits by the
oracle's elastic-net stop test and objective.
"""
import numpy as np
import pytest

from oracle import enet as EN
from oracle import fsqrppa as O
from paper_2601_02826_gb300 import synth
from tests.gpu_helpers import max_rel, memo, to_np

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


def _setup(seed=401, n=350, p=900, c=2):
    w = synth.tiny_geno(seed, n, p, c=c, fmt=1, G=4, taus=(0.5,))
    d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
    mu = O.default_mu(w.y)
    bp = w.block_ptr()
    eta = O.eta_blocks(d.Xt, bp, mu)
    return w, d, mu, bp, eta


@pytest.mark.parametrize("precision,slots,tol", [(0, 1, 1e-9), (1, 2, 1e-7), (1, 16, 1e-7)])
def test_enet_iterates_match_oracle(ctx, precision, slots, tol):
    from paper_2601_02826_gb300.device import upload
    w, d, mu, bp, eta = _setup()
    dw = upload(ctx, w)
    taus = [0.3, 0.6]
    lmaxs = [O.lambda_max(d.Xt, w.y, t, w.omega) for t in taus]
    lams = np.array([[0.25 * lm] for lm in lmaxs])
    gamma = 0.7 * lmaxs[0]
    B, N = 2, 50
    beta = torch.zeros(B * w.P, dtype=torch.float64, device="cuda")
    z = torch.zeros(B * w.n, dtype=torch.float64, device="cuda")
    th = torch.zeros(B * w.n, dtype=torch.float64, device="cuda")
    rc, infos = ctx.fit_batch(dw.design, dw.y, taus, lams, dw.omega, bp, beta, z, th,
                              opts=dict(tol=0.0, max_iter=N, mu=mu, eta=eta, precision=precision, max_group=slots,
                                        ridge=gamma))
    bb, zz, tt = to_np(beta).reshape(B, -1), to_np(z).reshape(B, -1), to_np(th).reshape(B, -1)
    for f, tau in enumerate(taus):
        lam = lams[f, 0] * w.omega
        ref = EN.fsqrppa_enet(d.Xt, w.y, tau, lam, gamma * w.omega, bp, eta, mu, tol=0.0, max_iter=N)
        assert max_rel(bb[f], ref.beta) <= tol
        assert max_rel(tt[f], ref.theta) <= tol
        assert max_rel(zz[f], ref.z) <= tol


@pytest.mark.parametrize("precision", [0, 1])
def test_enet_converged_fit_matches_oracle(ctx, precision):
    from paper_2601_02826_gb300.device import upload
    w, d, mu, bp, eta = _setup(402, 300, 400, 1)
    dw = upload(ctx, w)
    tau = 0.4
    lmax = O.lambda_max(d.Xt, w.y, tau, w.omega)
    lam_s = 0.3 * lmax
    gamma = 1.5 * lmax
    lam, gam = lam_s * w.omega, gamma * w.omega
    ref = memo(("enet", tau), lambda: EN.fsqrppa_enet(d.Xt, w.y, tau, lam, gam, bp, eta, mu, tol=1e-7,
                                                      max_iter=900000, lam_norm=lmax))
    assert ref.converged
    b = torch.zeros(w.P, dtype=torch.float64, device="cuda")
    z = torch.zeros(w.n, dtype=torch.float64, device="cuda")
    th = torch.zeros(w.n, dtype=torch.float64, device="cuda")
    rc, info = ctx.fit(dw.design, dw.y, tau, lam_s, dw.omega, bp, b, z, th,
                       opts=dict(tol=1e-6, max_iter=900000, mu=mu, eta=eta, precision=precision, ridge=gamma))
    assert rc == 0
    bb, zz, tt = to_np(b), to_np(z), to_np(th)
    ko = EN.kkt(d.Xt, w.y, tau, lam, gam, lmax, bb, zz, tt)
    assert ko.value <= 1.001e-6, ko
    f_gpu = EN.objective(d.Xt, w.y, bb, tau, lam, gam)
    assert f_gpu == pytest.approx(EN.objective(d.Xt, w.y, ref.beta, tau, lam, gam), rel=1e-6)
    assert info.primal == pytest.approx(f_gpu, rel=1e-9)
    assert np.isnan(info.gap)
    pen = w.omega > 0
    assert np.max(np.abs(bb[pen] - ref.beta[pen])) <= 1e-5
