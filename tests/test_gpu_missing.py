"""Mean imputation of missing genotypes (Section 7.2: a missing entry takes
the column mean, standardised value 0) on the GPU against the oracle, which
forms X~ with the imputed zeros explicitly. int8 (any code above 2) and 2-bit
(code 3) storage, 1 % missing entries; every product of the path carries the
correction, so the set-up quantities, the iterates of every kernel path and
the converged fits all match.
"""
import numpy as np
import pytest

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


CASES = {
    "int8": lambda: synth.tiny_geno(601, 410, 1500, c=2, fmt=synth.FMT_INT8, G=4, missing=0.01, taus=(0.4,)),
    "2bit": lambda: synth.tiny_geno(602, 390, 1300, c=2, fmt=synth.FMT_2BIT, G=3, missing=0.01, taus=(0.6,)),
}


def _oracle(w):
    d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
    return d


@pytest.mark.parametrize("case", list(CASES))
def test_setup_quantities_with_missing_entries(ctx, case):
    from paper_2601_02826_gb300.device import upload
    w = CASES[case]()
    d = _oracle(w)
    assert (O.decode_stored(w.geno, w.fmt, w.n) < 0).mean() > 0.005
    dw = upload(ctx, w)
    m = torch.zeros(w.c + w.p, dtype=torch.float64, device="cuda")
    s = torch.zeros(w.c + w.p, dtype=torch.float64, device="cuda")
    ctx.col_stats(dw.design, m, s)
    assert max_rel(to_np(m), d.mean[1:]) <= 1e-12 and max_rel(to_np(s), d.sd[1:]) <= 1e-12
    for tau in (0.2, 0.6):
        assert ctx.lambda_max(dw.design, dw.y, tau, dw.omega) == pytest.approx(
            O.lambda_max(d.Xt, w.y, tau, w.omega), rel=1e-10)
    mu = O.default_mu(w.y)
    got = ctx.eta(dw.design, w.block_ptr(), mu, 0.05, 30, 0.0)
    ref = O.eta_blocks(d.Xt, w.block_ptr(), mu, 0.05, 30, 0.0)
    assert max_rel(got, ref) <= 1e-9
    # predictions x~^T beta of a dense beta touch every missing entry
    rng = np.random.default_rng(1)
    beta = rng.standard_normal(w.P)
    out = torch.zeros(w.n, dtype=torch.float64, device="cuda")
    ctx.predict(dw.design, torch.from_numpy(beta).cuda(), 1, out)
    assert max_rel(to_np(out), d.Xt @ beta) <= 1e-12


@pytest.mark.parametrize("case,precision,slots", [("int8", 0, 1), ("int8", 1, 3), ("int8", 1, 16), ("2bit", 0, 2)])
def test_iterates_with_missing_entries(ctx, case, precision, slots):
    from paper_2601_02826_gb300.device import upload
    w = CASES[case]()
    d = _oracle(w)
    taus = [0.3, 0.5, 0.7][:max(1, min(3, slots))]
    lmaxs = [O.lambda_max(d.Xt, w.y, t, w.omega) for t in taus]
    lams = np.array([[0.2 * lm] for lm in lmaxs])
    mu = O.default_mu(w.y)
    bp = w.block_ptr()
    eta = O.eta_blocks(d.Xt, bp, mu)
    B, N = len(taus), 40
    dw = upload(ctx, w)
    beta = torch.zeros(B * w.P, dtype=torch.float64, device="cuda")
    z = torch.zeros(B * w.n, dtype=torch.float64, device="cuda")
    th = torch.zeros(B * w.n, dtype=torch.float64, device="cuda")
    ctx.fit_batch(dw.design, dw.y, taus, lams, dw.omega, bp, beta, z, th,
                  opts=dict(tol=0.0, max_iter=N, mu=mu, eta=eta, precision=precision, max_group=slots))
    bb, zz, tt = to_np(beta).reshape(B, -1), to_np(z).reshape(B, -1), to_np(th).reshape(B, -1)
    tol = 1e-9 if precision == 0 else 1e-7
    for f, tau in enumerate(taus):
        ref = O.fsqrppa(d.Xt, w.y, tau, lams[f, 0] * w.omega, bp, eta, mu, tol=0.0, max_iter=N)
        assert max_rel(bb[f], ref.beta) <= tol, f
        assert max_rel(tt[f], ref.theta) <= tol, f
        assert max_rel(zz[f], ref.z) <= tol, f


@pytest.mark.parametrize("precision", [0, 1])
def test_converged_fit_with_missing_entries(ctx, precision):
    from paper_2601_02826_gb300.device import upload
    w = synth.tiny_geno(603, 300, 400, c=1, fmt=synth.FMT_INT8, G=3, missing=0.01, taus=(0.5,))
    d = _oracle(w)
    tau = 0.5
    lmax = O.lambda_max(d.Xt, w.y, tau, w.omega)
    lam = 0.3 * lmax
    mu = O.default_mu(w.y)
    eta = O.eta_blocks(d.Xt, w.block_ptr(), mu)
    dw = upload(ctx, w)
    b = torch.zeros(w.P, dtype=torch.float64, device="cuda")
    z = torch.zeros(w.n, dtype=torch.float64, device="cuda")
    th = torch.zeros(w.n, dtype=torch.float64, device="cuda")
    rc, info = ctx.fit(dw.design, dw.y, tau, lam, dw.omega, w.block_ptr(), b, z, th,
                       opts=dict(tol=1e-6, max_iter=900000, mu=mu, eta=eta, precision=precision))
    assert rc == 0
    bb, zz, tt = to_np(b), to_np(z), to_np(th)
    assert O.kkt(d.Xt, w.y, tau, lam * w.omega, lmax, bb, zz, tt).value <= 1.001e-6
    ref = memo(("missing", tau), lambda: O.fsqrppa(d.Xt, w.y, tau, lam * w.omega, w.block_ptr(), eta, mu,
                                                   tol=1e-6, max_iter=900000, lam_norm=lmax))
    assert O.objective(d.Xt, w.y, bb, tau, lam * w.omega) == pytest.approx(
        O.objective(d.Xt, w.y, ref.beta, tau, lam * w.omega), rel=1e-6)


def test_noalloc_entry_point_rejects_missing_entries(ctx):
    from paper_2601_02826_gb300 import fsqr
    from paper_2601_02826_gb300.device import upload
    w = CASES["int8"]()
    dw = upload(ctx, w)
    with pytest.raises(fsqr.FsqrError) as e:
        ctx.lambda_max_noalloc(dw.design, dw.y, 0.5, dw.omega)
    assert e.value.code == fsqr.EINVAL and "missing" in str(e.value)
