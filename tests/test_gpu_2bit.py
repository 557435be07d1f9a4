"""2-bit genotype storage on the tensor-core path (FSQR_MIXED) against the
FP64 oracle, through the C ABI. The column pass bulk-copies packed 4 KB
tiles and its decode warps expand them into the E4M3 operand; the X~ beta
pass expands the active columns' packed runs while gathering them. The
products stay exact integers, so the iterates track the oracle's FP64 run
to the 1e-7 of the theta rounding, as on int8 storage.
"""
import numpy as np
import pytest

from oracle import fsqrppa as O
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


CASES = {
    # several tiles, n not a multiple of 128 (a partial sample chunk), covariates
    "tiles": lambda: synth.tiny_geno(801, 1000, 3000, c=2, fmt=synth.FMT_2BIT, G=4, taus=(0.5,)),
    # more 128-column tiles than SMs, cut into sample slices at the tail
    "sliced": lambda: synth.tiny_geno(802, 700, 24576, c=1, fmt=synth.FMT_2BIT, G=6, taus=(0.5,)),
    # 1 % missing codes (mean imputation)
    "missing": lambda: synth.tiny_geno(803, 517, 2000, c=2, fmt=synth.FMT_2BIT, G=3, missing=0.01, taus=(0.5,)),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("nfits", [1, 3])
def test_2bit_tensor_core_iterates_match_oracle(ctx, case, nfits):
    from paper_2601_02826_gb300.device import upload
    w = CASES[case]()
    d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
    taus = [0.3, 0.5, 0.8][:nfits]
    lmaxs = [O.lambda_max(d.Xt, w.y, t, w.omega) for t in taus]
    lams = np.array([[0.2 * lm] for lm in lmaxs])
    mu = O.default_mu(w.y)
    bp = w.block_ptr()
    eta = O.eta_blocks(d.Xt, bp, mu)
    N = 30
    dw = upload(ctx, w)
    beta = torch.zeros(nfits * w.P, dtype=torch.float64, device="cuda")
    z = torch.zeros(nfits * w.n, dtype=torch.float64, device="cuda")
    th = torch.zeros(nfits * w.n, dtype=torch.float64, device="cuda")
    ctx.profile(enable=False, reset=True)
    ctx.fit_batch(dw.design, dw.y, taus, lams, dw.omega, bp, beta, z, th,
                  opts=dict(tol=0.0, max_iter=N, mu=mu, eta=eta, precision=1, max_group=nfits))
    assert ctx.profile().tc_groups >= 1
    bb, zz, tt = to_np(beta).reshape(nfits, -1), to_np(z).reshape(nfits, -1), to_np(th).reshape(nfits, -1)
    for f, tau in enumerate(taus):
        ref = O.fsqrppa(d.Xt, w.y, tau, lams[f, 0] * w.omega, bp, eta, mu, tol=0.0, max_iter=N)
        assert max_rel(bb[f], ref.beta) <= 1e-7, f
        assert max_rel(tt[f], ref.theta) <= 1e-7, f
        assert max_rel(zz[f], ref.z) <= 1e-7, f


def test_2bit_tensor_core_converged_fit(ctx):
    from paper_2601_02826_gb300.device import upload
    w = synth.tiny_geno(105, 300, 400, c=1, fmt=synth.FMT_2BIT, G=3, taus=(0.5,))
    d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
    tau = 0.25
    lmax = O.lambda_max(d.Xt, w.y, tau, w.omega)
    lam = 0.3 * lmax
    mu = O.default_mu(w.y)
    eta = O.eta_blocks(d.Xt, w.block_ptr(), mu)
    dw = upload(ctx, w)
    b = torch.zeros(w.P, dtype=torch.float64, device="cuda")
    z = torch.zeros(w.n, dtype=torch.float64, device="cuda")
    th = torch.zeros(w.n, dtype=torch.float64, device="cuda")
    rc, info = ctx.fit(dw.design, dw.y, tau, lam, dw.omega, w.block_ptr(), b, z, th,
                       opts=dict(tol=1e-6, max_iter=900000, mu=mu, eta=eta, precision=1))
    assert rc == 0
    bb, zz, tt = to_np(b), to_np(z), to_np(th)
    ko = O.kkt(d.Xt, w.y, tau, lam * w.omega, lmax, bb, zz, tt)
    assert ko.value <= 1.001e-6 and info.kkt >= ko.value * (1 - 1e-6)
    ref = O.fsqrppa(d.Xt, w.y, tau, lam * w.omega, w.block_ptr(), eta, mu, tol=1e-6, max_iter=900000, lam_norm=lmax)
    assert O.objective(d.Xt, w.y, bb, tau, lam * w.omega) == pytest.approx(
        O.objective(d.Xt, w.y, ref.beta, tau, lam * w.omega), rel=1e-6)
