"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Sizes span several column tiles and a ragged tail (n and P not multiples of
16/32, several CTAs of the column pass, several row chunks of the X~ beta
pass). Tolerances:
  * setup quantities (column stats, lambda_max, eta): 1e-9 relative
    (same definitions, different FP64 summation order);
  * FP64 iterates after N steps from the same start: 1e-9 relative;
  * converged fits: objective 1e-6 relative, beta 1e-5 max-abs, and the
    KKT of the GPU's output recomputed by the oracle <= the tolerance.
"""
import math

import numpy as np
import pytest

from oracle import fsqrppa as O
from paper_2601_02826_gb300 import synth
from tests.gpu_helpers import max_rel, memo, oracle_problem, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    "dense": lambda: synth.small_dense(seed=101, n=61, p=150, G=3, tau=0.5),
    "int8": lambda: synth.tiny_geno(112, 333, 1000, c=2, fmt=synth.FMT_INT8, G=5, taus=(0.3,)),
    "2bit": lambda: synth.tiny_geno(103, 257, 700, c=0, fmt=synth.FMT_2BIT, G=4, taus=(0.7,)),
    "rows": lambda: synth.tiny_geno(104, 2500, 300, c=1, fmt=synth.FMT_INT8, G=2, taus=(0.5,)),
}


@pytest.fixture(scope="module")
def ctx():
    from paper_2601_02826_gb300 import fsqr
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = fsqr.Context(0, torch.cuda.current_stream().cuda_stream)
    yield c
    c.close()


def _up(ctx, w):
    from paper_2601_02826_gb300.device import upload
    return upload(ctx, w)


@pytest.mark.parametrize("case", list(CASES))
def test_column_stats(ctx, case):
    w = CASES[case]()
    dw = _up(ctx, w)
    F = w.c + w.p
    m = torch.zeros(F, dtype=torch.float64, device="cuda")
    s = torch.zeros(F, dtype=torch.float64, device="cuda")
    ctx.col_stats(dw.design, m, s)
    d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
    assert max_rel(to_np(m), d.mean[1:]) <= 1e-12
    assert max_rel(to_np(s), d.sd[1:]) <= 1e-12


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("tau", [0.1, 0.5, 0.77])
def test_lambda_max(ctx, case, tau):
    w = CASES[case]()
    dw = _up(ctx, w)
    got = ctx.lambda_max(dw.design, dw.y, tau, dw.omega)
    d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
    ref = O.lambda_max(d.Xt, w.y, tau, w.omega)
    assert got == pytest.approx(ref, rel=1e-10)


@pytest.mark.parametrize("case", list(CASES))
def test_eta_power_method(ctx, case):
    w = CASES[case]()
    dw = _up(ctx, w)
    d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
    mu = O.default_mu(w.y)
    for it, tol in [(7, 0.0), (100, 1e-6)]:
        got = ctx.eta(dw.design, w.block_ptr(), mu, 0.05, it, tol)
        ref = O.eta_blocks(d.Xt, w.block_ptr(), mu, 0.05, it, tol)
        assert max_rel(got, ref) <= 1e-9, (it, got, ref)


def _run(ctx, dw, w, tau, lam, mu, eta, n_iter, start=None, precision=0, tol=0.0, K=10, **kw):
    beta = torch.zeros(w.P, dtype=torch.float64, device="cuda")
    z = torch.tensor(w.y, device="cuda").clone()
    theta = torch.zeros(w.n, dtype=torch.float64, device="cuda")
    warm = 0
    if start is not None:
        beta.copy_(torch.tensor(start[0]))
        z.copy_(torch.tensor(start[1]))
        theta.copy_(torch.tensor(start[2]))
        warm = 1
    opts = dict(tol=tol, max_iter=n_iter, check_every=K, mu=mu, eta=eta, precision=precision, warm=warm)
    opts.update(kw)
    rc, info = ctx.fit(dw.design, dw.y, tau, lam, dw.omega, w.block_ptr(), beta, z, theta, opts=opts)
    return rc, info, to_np(beta), to_np(z), to_np(theta)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("n_iter", [10, 60])
def test_fp64_iterates_match_oracle(ctx, case, n_iter):
    w = CASES[case]()
    tau = w.taus[0]
    d, lmax, lam_s, lam, mu, bp, eta = oracle_problem(w, tau, 0.2)
    dw = _up(ctx, w)
    rc, info, b, z, t = _run(ctx, dw, w, tau, lam_s, mu, eta, n_iter)
    ref = O.fsqrppa(d.Xt, w.y, tau, lam, bp, eta, mu, tol=0.0, max_iter=n_iter, lam_norm=lmax)
    assert info.iters == n_iter == ref.iters
    assert max_rel(b, ref.beta) <= 1e-9
    assert max_rel(z, ref.z) <= 1e-9
    assert max_rel(t, ref.theta) <= 1e-9
    # the stop-test residuals the kernels reduced for w^N
    assert info.kkt == pytest.approx(ref.kkt.value, rel=1e-7)
    assert info.r_beta == pytest.approx(ref.kkt.r_beta, rel=1e-7, abs=1e-15)


def test_warm_start_continues_the_iteration(ctx):
    """Checkpoint/resume: 2 x 30 steps from a returned iterate equal 60 steps."""
    w = CASES["int8"]()
    tau = w.taus[0]
    d, lmax, lam_s, lam, mu, bp, eta = oracle_problem(w, tau, 0.2)
    dw = _up(ctx, w)
    _, _, b1, z1, t1 = _run(ctx, dw, w, tau, lam_s, mu, eta, 30)
    _, _, b2, z2, t2 = _run(ctx, dw, w, tau, lam_s, mu, eta, 30, start=(b1, z1, t1))
    _, _, b3, z3, t3 = _run(ctx, dw, w, tau, lam_s, mu, eta, 60)
    assert np.array_equal(b2, b3) and np.array_equal(z2, z3) and np.array_equal(t2, t3)


@pytest.mark.parametrize("case,frac", [("dense", 0.3), ("int8", 0.3), ("2bit", 0.5)])
def test_fp64_converged_fit_matches_oracle(ctx, case, frac):
    w = CASES[case]()
    tau = w.taus[0]
    d, lmax, lam_s, lam, mu, bp, eta = oracle_problem(w, tau, frac)
    dw = _up(ctx, w)
    rc, info, b, z, t = _run(ctx, dw, w, tau, lam_s, mu, eta, 200000, tol=1e-6)
    assert rc == 0 and info.status == 0
    ref = memo(("parity", case, frac), lambda: O.fsqrppa(d.Xt, w.y, tau, lam, bp, eta, mu, tol=1e-6,
                                                         max_iter=200000, lam_norm=lmax))
    assert ref.converged
    assert abs(info.iters - ref.iters) <= 10
    ko = O.kkt(d.Xt, w.y, tau, lam, lmax, b, z, t)
    assert ko.value <= 1e-6 * (1 + 1e-6)
    assert O.objective(d.Xt, w.y, b, tau, lam) == pytest.approx(O.objective(d.Xt, w.y, ref.beta, tau, lam), rel=1e-6)
    assert np.max(np.abs(b - ref.beta)) <= 1e-5
    assert info.primal == pytest.approx(O.objective(d.Xt, w.y, b, tau, lam), rel=1e-10)
    assert info.active == int(np.sum(b[1:] != 0))


@pytest.mark.parametrize("precision,digits", [(1, 4), (2, 4), (2, 5)])
def test_mixed_converged_fit_matches_oracle(ctx, precision, digits):
    """precision 1: tensor-core digit products; 2: DP4A digit products."""
    w = CASES["int8"]()
    tau = w.taus[0]
    d, lmax, lam_s, lam, mu, bp, eta = oracle_problem(w, tau, 0.3)
    dw = _up(ctx, w)
    rc, info, b, z, t = _run(ctx, dw, w, tau, lam_s, mu, eta, 200000, tol=1e-6, precision=precision,
                             digits=digits)
    assert rc == 0
    ref = memo(("parity", "int8", 0.3), lambda: O.fsqrppa(d.Xt, w.y, tau, lam, bp, eta, mu, tol=1e-6,
                                                          max_iter=200000, lam_norm=lmax))
    ko = O.kkt(d.Xt, w.y, tau, lam, lmax, b, z, t)
    assert ko.value <= 1e-6 * (1 + 1e-3)
    assert O.objective(d.Xt, w.y, b, tau, lam) == pytest.approx(O.objective(d.Xt, w.y, ref.beta, tau, lam), rel=1e-6)
    assert np.max(np.abs(b - ref.beta)) <= 1e-5


@pytest.mark.parametrize("case", ["int8", "rows"])
@pytest.mark.parametrize("precision,digits", [(1, 4), (2, 5)])
def test_mixed_iterates_track_fp64(ctx, case, precision, digits):
    """The digit products differ from FP64 only by the theta quantisation
    (2^-28 of max |theta| for 7 base-16 digits, 2^-35 for 5 int8 digits)."""
    w = CASES[case]()
    tau = w.taus[0]
    d, lmax, lam_s, lam, mu, bp, eta = oracle_problem(w, tau, 0.2)
    dw = _up(ctx, w)
    _, _, b, z, t = _run(ctx, dw, w, tau, lam_s, mu, eta, 50, precision=precision, digits=digits)
    ref = O.fsqrppa(d.Xt, w.y, tau, lam, bp, eta, mu, tol=0.0, max_iter=50)
    assert max_rel(b, ref.beta) <= 1e-7
    assert max_rel(t, ref.theta) <= 1e-7


def test_mixed_iterates_track_fp64_sliced_tail(ctx):
    """More 128-column tiles (192) than SMs: each CTA takes a whole tile and the
    40 left over are cut into sample slices whose integer digit sums are added
    up by the last slice to finish (3 slices of 8 sample blocks: 2, 3, 3)."""
    w = synth.tiny_geno(113, 1000, 24576, c=2, fmt=synth.FMT_INT8, G=7, taus=(0.4,))
    tau = w.taus[0]
    d, lmax, lam_s, lam, mu, bp, eta = oracle_problem(w, tau, 0.2)
    dw = _up(ctx, w)
    _, _, b, z, t = _run(ctx, dw, w, tau, lam_s, mu, eta, 30, precision=1, digits=4)
    ref = O.fsqrppa(d.Xt, w.y, tau, lam, bp, eta, mu, tol=0.0, max_iter=30)
    assert max_rel(b, ref.beta) <= 1e-7
    assert max_rel(t, ref.theta) <= 1e-7
    assert max_rel(z, ref.z) <= 1e-7


def test_batch_of_eight_fits_on_tensor_cores(ctx):
    """8 fits (4 tau x 2 lambda) advanced together per X pass on the tensor
    cores: 56 digit rows of theta, 88 of the X~ beta weights."""
    w = synth.tiny_geno(106, 260, 700, c=2, fmt=synth.FMT_INT8, G=3, taus=(0.3,))
    dw = _up(ctx, w)
    d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
    taus = [0.15, 0.4, 0.6, 0.75]
    fr = [0.25, 0.1]  # the oracle needs 62k to 155k steps for these 8 fits
    lmaxs = [O.lambda_max(d.Xt, w.y, t, w.omega) for t in taus]
    lams = np.array([[f * lm for f in fr] for lm in lmaxs])
    B = 8
    beta = torch.zeros(B * w.P, dtype=torch.float64, device="cuda")
    z = torch.zeros(B * w.n, dtype=torch.float64, device="cuda")
    th = torch.zeros(B * w.n, dtype=torch.float64, device="cuda")
    rc, infos = ctx.fit_batch(dw.design, dw.y, taus, lams, dw.omega, w.block_ptr(), beta, z, th,
                              opts=dict(tol=1e-6, max_iter=1_000_000, precision=1, max_group=8))
    assert rc == 0
    bb, zz, tt = to_np(beta).reshape(B, -1), to_np(z).reshape(B, -1), to_np(th).reshape(B, -1)
    for t_i, tau in enumerate(taus):
        for l_i in range(len(fr)):
            f = t_i * len(fr) + l_i
            lam = lams[t_i, l_i] * w.omega
            assert O.kkt(d.Xt, w.y, tau, lam, lmaxs[t_i], bb[f], zz[f], tt[f]).value <= 1.001e-6, f


def test_autotuned_group_size(ctx):
    """max_group = 0: the group size is chosen by timing the candidates on the
    first fits; every fit still meets the oracle's stop test, and the choice
    is cached for the next call on the same shape."""
    w = synth.tiny_geno(107, 240, 600, c=1, fmt=synth.FMT_INT8, G=3, taus=(0.4,))
    dw = _up(ctx, w)
    d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
    taus = [0.3, 0.5, 0.7]
    fr = [0.6, 0.35]  # the oracle needs 26k to 212k steps for these 6 fits
    lmaxs = [O.lambda_max(d.Xt, w.y, t, w.omega) for t in taus]
    lams = np.array([[f * lm for f in fr] for lm in lmaxs])
    B = 6
    chosen = []
    for _ in range(2):
        beta = torch.zeros(B * w.P, dtype=torch.float64, device="cuda")
        z = torch.zeros(B * w.n, dtype=torch.float64, device="cuda")
        th = torch.zeros(B * w.n, dtype=torch.float64, device="cuda")
        ctx.profile(enable=False, reset=True)
        rc, infos = ctx.fit_batch(dw.design, dw.y, taus, lams, dw.omega, w.block_ptr(), beta, z, th,
                                  opts=dict(tol=1e-6, max_iter=1_000_000, precision=1, max_group=0))
        assert rc == 0
        chosen.append(ctx.profile(enable=False).tuned_group)
        bb, zz, tt = to_np(beta).reshape(B, -1), to_np(z).reshape(B, -1), to_np(th).reshape(B, -1)
        for t_i, tau in enumerate(taus):
            for l_i in range(len(fr)):
                f = t_i * len(fr) + l_i
                lam = lams[t_i, l_i] * w.omega
                assert O.kkt(d.Xt, w.y, tau, lam, lmaxs[t_i], bb[f], zz[f], tt[f]).value <= 1.001e-6, f
    assert chosen[0] in (1, 2, 3, 4, 6) and chosen[1] == chosen[0]


def test_batch_grid_and_path_warm_start(ctx):
    w = synth.tiny_geno(105, 300, 400, c=1, fmt=synth.FMT_INT8, G=3, taus=(0.25, 0.75))
    dw = _up(ctx, w)
    g = O.decode_stored(w.geno, w.fmt, w.n)
    d = O.build_design(g, w.cov)
    mu = O.default_mu(w.y)
    bp = w.block_ptr()
    eta = O.eta_blocks(d.Xt, bp, mu)
    taus = [0.25, 0.75]
    fr = [0.6, 0.3]
    lmaxs = [O.lambda_max(d.Xt, w.y, t, w.omega) for t in taus]
    lams = np.array([[f * lm for f in fr] for lm in lmaxs])
    B = len(taus) * len(fr)
    refs = {}
    for t_i, tau in enumerate(taus):
        for l_i in range(len(fr)):
            lam = lams[t_i, l_i] * w.omega
            refs[t_i, l_i] = O.fsqrppa(d.Xt, w.y, tau, lam, bp, eta, mu, tol=1e-6, max_iter=400000,
                                       lam_norm=lmaxs[t_i])
    for warm, prec in [(0, 0), (2, 0), (2, 1), (0, 2)]:
        beta = torch.zeros(B * w.P, dtype=torch.float64, device="cuda")
        z = torch.zeros(B * w.n, dtype=torch.float64, device="cuda")
        th = torch.zeros(B * w.n, dtype=torch.float64, device="cuda")
        rc, infos = ctx.fit_batch(dw.design, dw.y, taus, lams, dw.omega, bp, beta, z, th,
                                  opts=dict(tol=1e-6, max_iter=400000, mu=mu, eta=eta, warm=warm,
                                            precision=prec, max_group=3))
        assert rc == 0
        bb, zz, tt = to_np(beta).reshape(B, -1), to_np(z).reshape(B, -1), to_np(th).reshape(B, -1)
        for t_i, tau in enumerate(taus):
            for l_i in range(len(fr)):
                f = t_i * len(fr) + l_i
                lam = lams[t_i, l_i] * w.omega
                ko = O.kkt(d.Xt, w.y, tau, lam, lmaxs[t_i], bb[f], zz[f], tt[f])
                assert ko.value <= 1.001e-6, (warm, prec, f, ko)
                assert O.objective(d.Xt, w.y, bb[f], tau, lam) == pytest.approx(
                    O.objective(d.Xt, w.y, refs[t_i, l_i].beta, tau, lam), rel=1e-6)
                assert infos[f].status == 0 and infos[f].lambda_max == pytest.approx(lmaxs[t_i], rel=1e-10)


@pytest.mark.parametrize("precision", [0, 1])
def test_lambda_above_lambda_max_gives_the_intercept_only_fit(ctx, precision):
    """The degenerate end of the path: at lambda = 1.02 lambda_max every
    penalised coefficient is exactly 0 at the converged iterate (a nonzero one
    would leave R_beta near 0.02), and the objective is the intercept-only one
    at the sample tau-quantile."""
    w = CASES["int8"]()
    tau = 0.3
    d, lmax, lam_s, lam, mu, bp, eta = oracle_problem(w, tau, 1.02)
    dw = _up(ctx, w)
    rc, info, b, z, t = _run(ctx, dw, w, tau, lam_s, mu, eta, 400000, tol=1e-6, precision=precision)
    assert rc == 0
    assert np.all(b[1:] == 0.0)
    q = np.sort(w.y)[math.ceil(w.n * tau) - 1]
    b0 = np.zeros(w.P)
    b0[0] = q
    assert O.objective(d.Xt, w.y, b, tau, lam) == pytest.approx(O.objective(d.Xt, w.y, b0, tau, lam), rel=1e-6)
    assert O.kkt(d.Xt, w.y, tau, lam, lmax, b, z, t).value <= 1.001e-6


def test_kkt_entry_point_matches_oracle(ctx):
    w = CASES["int8"]()
    tau = w.taus[0]
    d, lmax, lam_s, lam, mu, bp, eta = oracle_problem(w, tau, 0.2)
    dw = _up(ctx, w)
    res = O.fsqrppa(d.Xt, w.y, tau, lam, bp, eta, mu, tol=0.0, max_iter=40)
    T = lambda a: torch.tensor(a, device="cuda")
    info = ctx.kkt(dw.design, dw.y, tau, lam_s, dw.omega, lmax, T(res.beta), T(res.z), T(res.theta))
    ref = O.kkt(d.Xt, w.y, tau, lam, lmax, res.beta, res.z, res.theta)
    for a, b in [(info.r_p, ref.r_p), (info.r_z, ref.r_z), (info.r_beta, ref.r_beta), (info.r_1, ref.r_1)]:
        assert a == pytest.approx(b, rel=1e-9, abs=1e-14)
    assert info.primal == pytest.approx(O.objective(d.Xt, w.y, res.beta, tau, lam), rel=1e-12)
    # gap needs every omega_j > 0 for j >= 1 (true for tiny_geno with penalised covariates)
    gap, P, D = O.duality_gap(d.Xt, w.y, tau, lam, res.beta, res.theta)
    assert info.dual == pytest.approx(D, rel=1e-8, abs=1e-12)
    assert info.gap == pytest.approx(gap, rel=1e-8, abs=1e-12)


def test_predict_and_back_transform(ctx):
    w = CASES["int8"]()
    dw = _up(ctx, w)
    d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
    rng = np.random.default_rng(0)
    B = 5
    beta = rng.normal(size=(B, w.P)) * (rng.random((B, w.P)) < 0.1)
    bt = torch.tensor(beta.ravel(), device="cuda")
    out = torch.zeros(B * w.n, dtype=torch.float64, device="cuda")
    ctx.predict(dw.design, bt, B, out)
    ref = (d.Xt @ beta.T).T
    assert max_rel(to_np(out).reshape(B, -1), ref) <= 1e-12
    bo = torch.zeros_like(bt)
    ctx.back_transform(dw.design, bt, B, bo)
    ref_bo = np.stack([O.back_transform(d, beta[b]) for b in range(B)])
    assert max_rel(to_np(bo).reshape(B, -1), ref_bo) <= 1e-12


def test_invalid_arguments_are_rejected_and_context_survives(ctx):
    from paper_2601_02826_gb300 import fsqr
    w = CASES["int8"]()
    dw = _up(ctx, w)
    st = lambda: (torch.zeros(w.P, dtype=torch.float64, device="cuda"),
                  torch.zeros(w.n, dtype=torch.float64, device="cuda"),
                  torch.zeros(w.n, dtype=torch.float64, device="cuda"))
    bp = w.block_ptr()
    bad = [
        dict(tau=0.0), dict(tau=1.0), dict(lam=-1.0), dict(bp=np.array([0, 5, 5, w.P])),
        dict(bp=np.array([0, w.P - 1])), dict(opts=dict(digits=9, precision=1)),
        dict(opts=dict(check_every=0)), dict(opts=dict(max_group=33)), dict(opts=dict(ridge=-1.0)),
    ]
    for case in bad:
        b, z, t = st()
        with pytest.raises(fsqr.FsqrError) as e:
            ctx.fit(dw.design, dw.y, case.get("tau", 0.5), case.get("lam", 0.1), dw.omega,
                    case.get("bp", bp), b, z, t, opts=case.get("opts"))
        assert e.value.code == fsqr.EINVAL
    om = dw.omega.clone()
    om[0] = 1.0
    b, z, t = st()
    with pytest.raises(fsqr.FsqrError):
        ctx.fit(dw.design, dw.y, 0.5, 0.1, om, bp, b, z, t)
    d2 = ctx.design(w.n, w.p, w.c, w.fmt, dw.geno, w.ld - 16, cov=dw.cov)
    with pytest.raises(fsqr.FsqrError):
        ctx.lambda_max(d2, dw.y, 0.5, dw.omega)
    # still usable
    assert ctx.lambda_max(dw.design, dw.y, 0.5, dw.omega) > 0


def test_missing_genotypes_are_imputed_not_misread(ctx):
    """Missing codes take the column mean (standardised value 0): lambda_max
    of a design with 2 % missing entries matches the oracle's imputation."""
    w = synth.tiny_geno(106, 200, 100, missing=0.02)
    dw = _up(ctx, w)
    d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
    assert np.isnan(O.raw_columns(O.decode_stored(w.geno, w.fmt, w.n), w.cov)).any()
    for tau in (0.3, 0.5):
        assert ctx.lambda_max(dw.design, dw.y, tau, dw.omega) == pytest.approx(
            O.lambda_max(d.Xt, w.y, tau, w.omega), rel=1e-10)


def test_timeout_returns_valid_iterate(ctx):
    w = CASES["rows"]()
    tau = w.taus[0]
    d, lmax, lam_s, lam, mu, bp, eta = oracle_problem(w, tau, 0.05)
    dw = _up(ctx, w)
    rc, info, b, z, t = _run(ctx, dw, w, tau, lam_s, mu, eta, 10_000_000, tol=1e-14, timeout_ms=200)
    assert rc == 3 and info.status == 3
    assert np.all(np.isfinite(b)) and np.all(np.isfinite(t)) and info.iters > 0


def test_max_iter_reports_noconv(ctx):
    w = CASES["dense"]()
    tau = 0.5
    d, lmax, lam_s, lam, mu, bp, eta = oracle_problem(w, tau, 0.1)
    dw = _up(ctx, w)
    rc, info, b, z, t = _run(ctx, dw, w, tau, lam_s, mu, eta, 20, tol=1e-12)
    assert rc == 2 and info.status == 2 and info.iters == 20
