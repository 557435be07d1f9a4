"""Path selection statistics and interval coverage (Section 7, 7.1) on the GPU
against oracle/select.py, through the C ABI, on seeded coefficient vectors
(sparse, so both the loss and the active count matter) and on a converged
path.
"""
import numpy as np
import pytest

from oracle import fsqrppa as O
from oracle import select as S
from paper_2601_02826_gb300 import synth
from tests.gpu_helpers import to_np

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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _betas(rng, B, P, k):
    out = np.zeros((B, P))
    for b in range(B):
        out[b, 0] = rng.standard_normal()
        idx = rng.choice(np.arange(1, P), size=min(k + b, P - 1), replace=False)
        out[b, idx] = 0.3 * rng.standard_normal(len(idx))
    return out


@pytest.mark.parametrize("fmt", [1, 2])
def test_path_stats_match_oracle_on_training_and_validation_data(ctx, fmt):
    from paper_2601_02826_gb300.device import upload
    w = synth.tiny_geno(301, 777, 2100, c=3, fmt=fmt, G=4, taus=(0.5,))
    v = synth.tiny_geno(302, 333, 2100, c=3, fmt=fmt, G=4, taus=(0.5,))
    d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
    rng = np.random.default_rng(5)
    B = 7
    betas = _betas(rng, B, w.P, 9)
    taus = list(np.linspace(0.1, 0.9, B))
    dw = upload(ctx, w)
    loss, act, hb = ctx.path_stats(dw.design, dw.y, taus, _dev(betas.ravel()))
    for b in range(B):
        assert loss[b] == pytest.approx(S.pinball_sum(d.Xt, w.y, betas[b], taus[b]) / w.n, rel=1e-12)
        assert act[b] == S.active_count(betas[b])
        assert hb[b] == pytest.approx(S.hbic(d.Xt, w.y, betas[b], taus[b], w.P - 1), rel=1e-12)
    # validation data standardised with the training columns' statistics
    Xv = S.standardise_with(d, O.decode_stored(v.geno, v.fmt, v.n), v.cov)
    gv = torch.from_numpy(np.ascontiguousarray(v.geno).view(np.uint8)).cuda()
    cv = _dev(v.cov)
    dv = ctx.design(v.n, v.p, v.c, v.fmt, gv, v.ld, cov=cv, col_mean=_dev(d.mean[1:]), col_sd=_dev(d.sd[1:]))
    vloss, _, _ = ctx.path_stats(dv, _dev(v.y), taus, _dev(betas.ravel()))
    for b in range(B):
        assert vloss[b] == pytest.approx(S.validation_loss(Xv, v.y, betas[b], taus[b]), rel=1e-12)
    assert S.select(vloss) == S.select([S.validation_loss(Xv, v.y, betas[b], taus[b]) for b in range(B)])


def test_interval_coverage_matches_oracle(ctx):
    from paper_2601_02826_gb300.device import upload
    w = synth.tiny_geno(303, 1000, 600, c=2, fmt=1, G=3, taus=(0.5,))
    d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
    rng = np.random.default_rng(6)
    lo, hi = _betas(rng, 2, w.P, 20)
    lo[0] -= 1.0
    hi[0] += 1.0  # mostly ordered, with some crossings left
    dw = upload(ctx, w)
    cov, wid, cr = ctx.interval_coverage(dw.design, dw.y, _dev(lo), _dev(hi))
    c0, w0, r0 = S.interval_coverage(d.Xt, w.y, lo, hi)
    assert cov == pytest.approx(c0, abs=0) and cr == r0 and wid == pytest.approx(w0, rel=1e-12)
    assert 0 < r0 < w.n


def test_hbic_selects_the_same_lambda_as_the_oracle_on_a_converged_path(ctx):
    """A path of 6 lambdas solved on the GPU (FP64) to KKT <= 1e-6: the
    oracle's HBIC of the GPU's fits picks the same index as the GPU's."""
    from paper_2601_02826_gb300.device import upload
    w = synth.tiny_geno(105, 300, 400, c=1, fmt=1, G=3, taus=(0.5,))
    dw = upload(ctx, w)
    d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
    tau = 0.25
    fr = [0.6, 0.45, 0.3, 0.2, 0.15, 0.1]
    lmax = O.lambda_max(d.Xt, w.y, tau, w.omega)
    lams = np.array([[f * lmax for f in fr]])
    B = len(fr)
    beta = torch.zeros(B * w.P, dtype=torch.float64, device="cuda")
    z = torch.zeros(B * w.n, dtype=torch.float64, device="cuda")
    th = torch.zeros(B * w.n, dtype=torch.float64, device="cuda")
    rc, _ = ctx.fit_batch(dw.design, dw.y, [tau], lams, dw.omega, w.block_ptr(), beta, z, th,
                          opts=dict(tol=1e-6, max_iter=900000, precision=0, max_group=3))
    assert rc == 0
    bb = to_np(beta).reshape(B, -1)
    _, act, hb = ctx.path_stats(dw.design, dw.y, [tau] * B, beta)
    ref = [S.hbic(d.Xt, w.y, bb[b], tau, w.P - 1) for b in range(B)]
    assert np.allclose(hb, ref, rtol=1e-12)
    assert S.select(hb) == S.select(ref)
    assert list(act) == [S.active_count(bb[b]) for b in range(B)]
