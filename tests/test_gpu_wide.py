"""Wide slot groups (16 or 32 fits per X pass on the tensor cores) against the
FP64 oracle, through the C ABI.

Every fit of a wide solve takes the steps of Algorithm 1 alone, from the step
at which it enters its slot; only the X pass is shared. So each fit's
iterates after N steps match the oracle's run of that fit (1e-7 relative, the
bound of the 28-bit theta rounding used in the other mixed tests), whatever
slot it ran in and whichever fits ran beside it; converged fits meet the
oracle's stop test; with more fits than slots, the slots are refilled.
"""
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


def _grid(w, taus, fracs):
    d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
    lmaxs = [O.lambda_max(d.Xt, w.y, t, w.omega) for t in taus]
    lams = np.array([[f * lm for f in fracs] for lm in lmaxs])
    return d, lmaxs, lams


def _solve(ctx, dw, w, taus, lams, opts):
    B = lams.size
    beta = torch.zeros(B * w.P, dtype=torch.float64, device="cuda")
    z = torch.zeros(B * w.n, dtype=torch.float64, device="cuda")
    th = torch.zeros(B * w.n, dtype=torch.float64, device="cuda")
    rc, infos = ctx.fit_batch(dw.design, dw.y, taus, lams, dw.omega, w.block_ptr(), beta, z, th, opts=opts)
    return rc, infos, to_np(beta).reshape(B, -1), to_np(z).reshape(B, -1), to_np(th).reshape(B, -1)


@pytest.mark.parametrize("slots,B", [(16, 12), (32, 20), (16, 21)])
def test_wide_iterates_match_oracle(ctx, slots, B):
    """B fits, N = 40 steps each (tolerance 0): with B > slots the later fits
    enter freed slots at a later global step, and still take their own 40."""
    from paper_2601_02826_gb300.device import upload
    w = synth.tiny_geno(201, 520, 3000, c=2, fmt=synth.FMT_INT8, G=4, taus=(0.5,))
    dw = upload(ctx, w)
    n_tau = 3 if B % 3 == 0 else (4 if B % 4 == 0 else 7)
    taus = list(np.linspace(0.15, 0.85, n_tau))
    fracs = list(np.geomspace(0.6, 0.1, B // n_tau))
    d, lmaxs, lams = _grid(w, taus, fracs)
    mu = O.default_mu(w.y)
    bp = w.block_ptr()
    eta = O.eta_blocks(d.Xt, bp, mu)
    N = 40
    rc, infos, bb, zz, tt = _solve(ctx, dw, w, taus, lams,
                                   dict(tol=0.0, max_iter=N, mu=mu, eta=eta, precision=1, max_group=slots))
    assert ctx.profile().wide_groups >= 1
    for t_i, tau in enumerate(taus):
        for l_i in range(len(fracs)):
            f = t_i * len(fracs) + l_i
            lam = lams[t_i, l_i] * w.omega
            ref = O.fsqrppa(d.Xt, w.y, tau, lam, bp, eta, mu, tol=0.0, max_iter=N)
            assert infos[f].iters == N, (f, infos[f].iters)
            assert max_rel(bb[f], ref.beta) <= 1e-7, f
            assert max_rel(tt[f], ref.theta) <= 1e-7, f
            assert max_rel(zz[f], ref.z) <= 1e-7, f


@pytest.mark.parametrize("warm", [0, 2])
def test_wide_converged_fits_meet_the_oracle_stop_test(ctx, warm):
    """18 fits (9 tau x 2 lambda) through 16 slots to KKT <= 1e-6, so two
    fits enter freed slots; with the path warm start (warm = 2) a fit starts
    from its predecessor's solution once that one has stopped. Objectives
    agree with the oracle's fits."""
    from paper_2601_02826_gb300.device import upload
    w = synth.tiny_geno(105, 300, 400, c=1, fmt=synth.FMT_INT8, G=3, taus=(0.5,))
    dw = upload(ctx, w)
    taus = [0.1, 0.2, 0.25, 0.35, 0.45, 0.5, 0.6, 0.75, 0.9]
    fracs = [0.6, 0.15]  # the oracle needs 26k to 112k steps for these
    d, lmaxs, lams = _grid(w, taus, fracs)
    mu = O.default_mu(w.y)
    bp = w.block_ptr()
    eta = O.eta_blocks(d.Xt, bp, mu)
    rc, infos, bb, zz, tt = _solve(ctx, dw, w, taus, lams,
                                   dict(tol=1e-6, max_iter=900000, mu=mu, eta=eta, precision=1, max_group=16,
                                        warm=warm))
    assert rc == 0, [i.status for i in infos]
    for t_i, tau in enumerate(taus):
        for l_i in range(len(fracs)):
            f = t_i * len(fracs) + l_i
            lam = lams[t_i, l_i] * w.omega
            ko = O.kkt(d.Xt, w.y, tau, lam, lmaxs[t_i], bb[f], zz[f], tt[f])
            assert ko.value <= 1.001e-6, (f, ko)
            assert infos[f].kkt >= ko.value * (1 - 1e-6), f  # the certified test is an upper bound
            if l_i == 1 and t_i in (0, 4, 8):
                val = O.objective(d.Xt, w.y, bb[f], tau, lam)
                if warm == 0:  # the oracle's cold run of the same fit
                    ref = O.fsqrppa(d.Xt, w.y, tau, lam, bp, eta, mu, tol=1e-6, max_iter=900000,
                                    lam_norm=lmaxs[t_i])
                    assert val == pytest.approx(O.objective(d.Xt, w.y, ref.beta, tau, lam), rel=1e-6)
                else:
                    # another start ends at another point of the KKT <= 1e-6 set, so the check
                    # is against the exact optimum (the LP); the oracle's own fits of these three
                    # problems, cold and path-started, sit 4.5e-6 to 8.2e-6 above it
                    _, opt = lp_solve(d.Xt, w.y, tau, lam)
                    assert opt - 1e-9 <= val <= opt * (1 + 2e-5) + 1e-12


def test_wide_max_iter_and_report(ctx):
    """Fits that hit max_iter stop with FSQR_ENOCONV and report their own
    iteration count; the primal value matches the oracle's objective."""
    from paper_2601_02826_gb300 import fsqr
    from paper_2601_02826_gb300.device import upload
    w = synth.tiny_geno(203, 200, 700, c=0, fmt=synth.FMT_INT8, G=2, taus=(0.5,))
    dw = upload(ctx, w)
    taus = [0.3, 0.7]
    fracs = [0.5, 0.3, 0.2]
    d, lmaxs, lams = _grid(w, taus, fracs)
    rc, infos, bb, zz, tt = _solve(ctx, dw, w, taus, lams, dict(tol=1e-12, max_iter=100, precision=1, max_group=32))
    assert rc == fsqr.ENOCONV
    for t_i, tau in enumerate(taus):
        for l_i in range(len(fracs)):
            f = t_i * len(fracs) + l_i
            assert infos[f].status == fsqr.ENOCONV and infos[f].iters == 100
            lam = lams[t_i, l_i] * w.omega
            assert infos[f].primal == pytest.approx(O.objective(d.Xt, w.y, bb[f], tau, lam), rel=1e-9)
