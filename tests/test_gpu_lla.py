"""L-step LLA for SCAD and MCP (Section 6, Algorithm 2) on the GPU against the
oracle (oracle/lla.py), through the C ABI.

The GPU and the oracle each run the weighted-l1 fit, reweight by p'_lambda of
their own solution and re-solve from it. The checks: the first fits agree
(objective 1e-6 relative); the weights the GPU used (lam_out) are the
oracle's formula applied to the GPU's first fit; the final iterate meets the
oracle's stop test for those weights; and the final concave objective and
support agree with the oracle's LLA fit.
"""
import numpy as np
import pytest

from oracle import fsqrppa as O
from oracle import lla as LLA
from paper_2601_02826_gb300 import synth
from tests.gpu_helpers import memo, to_np

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


@pytest.mark.parametrize("penalty,a,precision", [("scad", 3.7, 0), ("mcp", 3.0, 0), ("scad", 3.7, 1)])
def test_one_step_lla_matches_oracle(ctx, penalty, a, precision):
    from paper_2601_02826_gb300 import fsqr
    from paper_2601_02826_gb300.device import upload
    w = synth.tiny_geno(105, 300, 400, c=1, fmt=synth.FMT_INT8, G=3, taus=(0.5,))
    dw = upload(ctx, w)
    tau, frac = 0.25, 0.3
    d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
    lmax = O.lambda_max(d.Xt, w.y, tau, w.omega)
    lam = frac * lmax
    mu = O.default_mu(w.y)
    bp = w.block_ptr()
    eta = O.eta_blocks(d.Xt, bp, mu)
    steps, weights = memo(("lla", penalty, a), lambda: LLA.lla_fit(d.Xt, w.y, tau, lam, w.omega, bp, eta, mu,
                                                                   penalty, a, L=1, tol=1e-6, max_iter=900000,
                                                                   lam_norm=lmax))
    assert all(s.converged for s in steps)
    # the GPU's first step alone
    b0 = torch.zeros(w.P, dtype=torch.float64, device="cuda")
    z0 = torch.zeros(w.n, dtype=torch.float64, device="cuda")
    t0 = torch.zeros(w.n, dtype=torch.float64, device="cuda")
    opts = dict(tol=1e-6, max_iter=900000, mu=mu, eta=eta, precision=precision)
    rc, _ = ctx.fit(dw.design, dw.y, tau, lam, dw.omega, bp, b0, z0, t0, opts=opts)
    assert rc == 0
    beta0 = to_np(b0)
    assert O.objective(d.Xt, w.y, beta0, tau, lam * w.omega) == pytest.approx(
        O.objective(d.Xt, w.y, steps[0].beta, tau, lam * w.omega), rel=1e-6)
    # the full LLA on the GPU
    pen = {"scad": fsqr.PEN_SCAD, "mcp": fsqr.PEN_MCP}[penalty]
    b = torch.zeros(w.P, dtype=torch.float64, device="cuda")
    z = torch.zeros(w.n, dtype=torch.float64, device="cuda")
    th = torch.zeros(w.n, dtype=torch.float64, device="cuda")
    lo = torch.zeros(w.P, dtype=torch.float64, device="cuda")
    rc, info = ctx.fit_lla(dw.design, dw.y, tau, lam, dw.omega, bp, pen, a, 1, b, z, th, lam_out=lo, opts=opts)
    assert rc == 0 and info.status == 0
    bl, zl, tl, wl = to_np(b), to_np(z), to_np(th), to_np(lo)
    w_expect = LLA.lla_weights(beta0, lam, w.omega, penalty, a)
    assert np.max(np.abs(wl - w_expect)) <= 1e-12 * lam
    ko = O.kkt(d.Xt, w.y, tau, wl, lmax, bl, zl, tl)
    assert ko.value <= 1.001e-6, ko
    f_gpu = LLA.concave_objective(d.Xt, w.y, bl, tau, lam, w.omega, penalty, a)
    f_ref = LLA.concave_objective(d.Xt, w.y, steps[1].beta, tau, lam, w.omega, penalty, a)
    assert f_gpu == pytest.approx(f_ref, rel=1e-5)
    assert set(np.flatnonzero(np.abs(bl[1:]) > 1e-6)) == set(np.flatnonzero(np.abs(steps[1].beta[1:]) > 1e-6))


def test_lla_rejects_bad_arguments(ctx):
    from paper_2601_02826_gb300 import fsqr
    from paper_2601_02826_gb300.device import upload
    w = synth.tiny_geno(105, 60, 40, c=0, fmt=synth.FMT_INT8, G=2, taus=(0.5,))
    dw = upload(ctx, w)
    b = torch.zeros(w.P, dtype=torch.float64, device="cuda")
    z = torch.zeros(w.n, dtype=torch.float64, device="cuda")
    th = torch.zeros(w.n, dtype=torch.float64, device="cuda")
    for pen, a in [(fsqr.PEN_SCAD, 2.0), (fsqr.PEN_MCP, 1.0), (7, 3.0)]:
        with pytest.raises(fsqr.FsqrError) as e:
            ctx.fit_lla(dw.design, dw.y, 0.5, 0.1, dw.omega, w.block_ptr(), pen, a, 1, b, z, th)
        assert e.value.code == fsqr.EINVAL
