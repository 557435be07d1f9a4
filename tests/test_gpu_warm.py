"""Learned warm start on the GPU against the FP64 oracle of oracle/mlp.py.

The network's kernels run in FP32, so they are compared with the FP64
oracle at FP32 tolerances. The forward pass is checked to 1e-5 relative, and
the gradient to 1e-4 relative to its largest entry. Batch sampling follows
the published splitmix64 definition on both sides. The starting point
(features, beta, z, theta) is compared with the oracle's. The fit solved from
that start must meet the same stop test as a cold fit.
"""
import numpy as np
import pytest

from oracle import fsqrppa as O
from oracle import mlp as M
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


def _f32(a):
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")


def _params(seed, scale=1.0):
    """Random parameters with He-scaled weights (numpy, float32-representable)."""
    rng = np.random.default_rng(seed)
    parts = []
    for a, b in zip(M.DIMS[:-1], M.DIMS[1:]):
        parts.append(rng.normal(0.0, scale * np.sqrt(2.0 / a), a * b))
        parts.append(rng.normal(0.0, 0.1, b))
    return np.concatenate(parts).astype(np.float32).astype(np.float64)


def test_param_count(ctx):
    assert ctx.mlp_param_count() == M.param_count()


def test_forward_matches_oracle(ctx):
    p = _params(1)
    x = np.random.default_rng(2).uniform(-1, 1, (1001, 3)).astype(np.float32).astype(np.float64)
    out = torch.zeros(1001, dtype=torch.float32, device="cuda")
    ctx.mlp_forward(_f32(p), _f32(x), out)
    ref, _ = M.forward(p, x)
    got = to_np(out).astype(np.float64)
    assert np.max(np.abs(got - ref)) <= 1e-5 * (1.0 + np.max(np.abs(ref)))


def test_gradient_matches_oracle(ctx):
    p = _params(3)
    rng = np.random.default_rng(4)
    rows = 777
    x = rng.uniform(-1, 1, (rows, 3)).astype(np.float32).astype(np.float64)
    t = rng.normal(0, 1, rows).astype(np.float32).astype(np.float64)
    w = rng.uniform(0.5, 3.0, rows).astype(np.float32).astype(np.float64)
    g = torch.zeros(M.param_count(), dtype=torch.float32, device="cuda")
    loss = ctx.mlp_grad(_f32(p), _f32(x), _f32(t), _f32(w), g)
    L, ref = M.grad(p, x, t, w)
    assert loss == pytest.approx(L, rel=1e-5)
    got = to_np(g).astype(np.float64)
    assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref))


def _splitmix64(x):
    """splitmix64 (Steele, Lea and Flood, 2014) on numpy uint64."""
    with np.errstate(over="ignore"):
        x = (x + np.uint64(0x9E3779B97F4A7C15)).astype(np.uint64)
        x = ((x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)).astype(np.uint64)
        x = ((x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)).astype(np.uint64)
        return x ^ (x >> np.uint64(31))


def test_one_training_step_matches_oracle_adam(ctx):
    p = _params(5)
    rng = np.random.default_rng(6)
    rows, batch, seed, lr = 500, 256, 12345, 1e-3
    x = rng.uniform(-1, 1, (rows, 3)).astype(np.float32).astype(np.float64)
    t = rng.normal(0, 1, rows).astype(np.float32).astype(np.float64)
    w = np.ones(rows)
    dp, dm, dv = _f32(p), torch.zeros(len(p), device="cuda"), torch.zeros(len(p), device="cuda")
    losses = ctx.mlp_train(dp, dm, dv, 0, _f32(x), _f32(t), _f32(w), 1, batch, lr, seed)
    # the batch of step 1, drawn as the header defines it
    with np.errstate(over="ignore"):
        k = np.uint64(1)
        h0 = _splitmix64(np.uint64(seed) ^ (k * np.uint64(0xD1B54A32D192ED03)))
        idx = (_splitmix64(h0 + np.arange(batch, dtype=np.uint64)) % np.uint64(rows)).astype(np.int64)
    L, g = M.grad(p, x[idx], t[idx], w[idx])
    assert losses[0] == pytest.approx(L, rel=1e-5)
    newp, _, _ = M.adam_step(p, g, np.zeros_like(p), np.zeros_like(p), 1, lr)
    got = to_np(dp).astype(np.float64)
    # a first Adam step moves each parameter by lr * g / (|g| + eps): compare
    # where the gradient is well above FP32 noise
    big = np.abs(g) > 1e-3 * np.max(np.abs(g))
    assert np.all(np.abs((got - p)[big] - (newp - p)[big]) <= 1e-3 * lr + 1e-6 * np.abs(p[big]))


def _up(ctx, w):
    from paper_2601_02826_gb300.device import upload
    return upload(ctx, w)


@pytest.mark.parametrize("tau,frac", [(0.3, 0.5), (0.7, 0.2)])
def test_features_and_start_match_oracle(ctx, tau, frac):
    w = synth.tiny_geno(141, 400, 900, c=2, fmt=synth.FMT_INT8, G=3, taus=(tau,))
    dw = _up(ctx, w)
    d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
    u = torch.zeros((w.P - 1, 3), dtype=torch.float32, device="cuda")
    lmax = ctx.warm_features(dw.design, dw.y, tau, frac, dw.omega, u)
    ref_u, ref_l = M.features(d.Xt, w.y, tau, frac, w.omega)
    assert lmax == pytest.approx(ref_l, rel=1e-10)
    assert np.max(np.abs(to_np(u) - ref_u)) <= 1e-6
    p = _params(7, scale=0.5)
    beta = torch.zeros(w.P, dtype=torch.float64, device="cuda")
    z = torch.zeros(w.n, dtype=torch.float64, device="cuda")
    th = torch.zeros(w.n, dtype=torch.float64, device="cuda")
    ctx.warm_start(dw.design, dw.y, tau, frac, dw.omega, _f32(p), beta, z, th)
    # the oracle evaluated on the float32 inputs the kernels saw
    f, _ = M.forward(p, to_np(u).astype(np.float64))
    rb = np.concatenate([[np.sort(w.y)[int(np.ceil(w.n * tau)) - 1]], np.std(w.y) * f])
    b = to_np(beta)
    assert np.max(np.abs(b - rb)) <= 1e-5 * (1.0 + np.max(np.abs(rb)))
    zz = to_np(z)
    np.testing.assert_allclose(zz, w.y - d.Xt @ b, rtol=0, atol=1e-9 * (1 + np.max(np.abs(w.y))))
    np.testing.assert_array_equal(to_np(th), (tau - (zz < 0)) / w.n)


def _fits_along_grid(ctx, dw, w, taus, fracs):
    """The solver's own solutions on a tau x lambda grid (FP64 path); rows of
    fits that did not reach KKT <= 1e-6 within the iteration cap are None."""
    d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
    lmaxs = [O.lambda_max(d.Xt, w.y, t, w.omega) for t in taus]
    lams = np.array([[f * lm for f in fracs] for lm in lmaxs])
    B = len(taus) * len(fracs)
    beta = torch.zeros(B * w.P, dtype=torch.float64, device="cuda")
    z = torch.zeros(B * w.n, dtype=torch.float64, device="cuda")
    th = torch.zeros(B * w.n, dtype=torch.float64, device="cuda")
    _, infos = ctx.fit_batch(dw.design, dw.y, taus, lams, dw.omega, w.block_ptr(), beta, z, th,
                             opts=dict(tol=1e-6, max_iter=300_000, max_group=8))
    bb = to_np(beta).reshape(B, w.P)
    return [bb[f] if infos[f].status == 0 else None for f in range(B)]


def test_learned_warm_start_keeps_the_fit_and_saves_iterations(ctx):
    """Trains the network on the solver's solutions for 3 problems, then solves
    4 fits of 2 held-out problems from a cold start and from the learned start.
    Fits that meet the stop test are checked again by the oracle, and where both
    starts converge their objectives agree. Counting a fit that hits the
    iteration cap as the cap, the learned start needs fewer iterations in total."""
    taus = [0.25, 0.5, 0.75]
    fracs = [0.6, 0.45, 0.35, 0.25]
    U, T, W = [], [], []
    for seed in (201, 202, 203):
        w = synth.tiny_geno(seed, 300, 800, c=0, fmt=synth.FMT_INT8, G=4)
        dw = _up(ctx, w)
        betas = _fits_along_grid(ctx, dw, w, taus, fracs)
        sdy = float(np.std(w.y))
        for ti, tau in enumerate(taus):
            for fi, fr in enumerate(fracs):
                b = betas[ti * len(fracs) + fi]
                if b is None:
                    continue
                u = torch.zeros((w.P - 1, 3), dtype=torch.float32, device="cuda")
                ctx.warm_features(dw.design, dw.y, tau, fr, dw.omega, u)
                t = b[1:] / sdy
                U.append(to_np(u))
                T.append(t)
                W.append(np.where(t != 0.0, 10.0, 1.0))
    assert len(U) >= 12
    U, T, W = np.concatenate(U), np.concatenate(T), np.concatenate(W)
    npar = ctx.mlp_param_count()
    params = torch.zeros(npar, dtype=torch.float32, device="cuda")
    ctx.mlp_init(params, 7)
    m = torch.zeros(npar, dtype=torch.float32, device="cuda")
    v = torch.zeros(npar, dtype=torch.float32, device="cuda")
    losses = ctx.mlp_train(params, m, v, 0, _f32(U), _f32(T), _f32(W), 2000, 4096, 1e-3, 11)
    assert np.mean(losses[-100:]) < 0.5 * np.mean(losses[:100])

    # a fit that does not reach the tolerance within the cap counts as the cap
    cap = 400_000
    cold_it, warm_it, both = 0, 0, 0
    report = []
    for seed in (301, 302):
        w = synth.tiny_geno(seed, 300, 800, c=0, fmt=synth.FMT_INT8, G=4)
        dw = _up(ctx, w)
        d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
        for tau, fr in [(0.35, 0.45), (0.6, 0.35)]:
            lmax = O.lambda_max(d.Xt, w.y, tau, w.omega)
            lam = fr * lmax * w.omega
            outs = []
            for learned in (False, True):
                beta = torch.zeros(w.P, dtype=torch.float64, device="cuda")
                z = torch.tensor(w.y, device="cuda").clone()
                th = torch.zeros(w.n, dtype=torch.float64, device="cuda")
                if learned:
                    ctx.warm_start(dw.design, dw.y, tau, fr, dw.omega, params, beta, z, th)
                rc, info = ctx.fit(dw.design, dw.y, tau, fr * lmax, dw.omega, w.block_ptr(), beta, z, th,
                                   opts=dict(tol=1e-6, max_iter=cap, warm=1 if learned else 0))
                ok = rc == 0
                b, zz, tt = to_np(beta), to_np(z), to_np(th)
                if ok:
                    assert O.kkt(d.Xt, w.y, tau, lam, lmax, b, zz, tt).value <= 1.001e-6
                outs.append((info.iters if ok else cap, O.objective(d.Xt, w.y, b, tau, lam), ok))
            (ci, co, cok), (wi, wo, wok) = outs
            if cok and wok:
                assert wo == pytest.approx(co, rel=1e-5)
                both += 1
            cold_it += ci
            warm_it += wi
            report.append((seed, tau, fr, ci, wi))
    print("learned warm start: (seed, tau, frac, cold iters, learned iters)", report,
          f"total {cold_it} -> {warm_it} ({warm_it / cold_it:.3f}x)")
    assert both >= 2
    assert warm_it < cold_it

    # the same start requested through fsqr_fit_batch (FSQR_WARM_LEARNED)
    w = synth.tiny_geno(301, 300, 800, c=0, fmt=synth.FMT_INT8, G=4)
    dw = _up(ctx, w)
    d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
    taus2, fr2 = [0.35, 0.6], [0.6, 0.45]
    lmaxs = [O.lambda_max(d.Xt, w.y, t, w.omega) for t in taus2]
    lams = np.array([[f * lm for f in fr2] for lm in lmaxs])
    beta = torch.zeros(4 * w.P, dtype=torch.float64, device="cuda")
    z = torch.zeros(4 * w.n, dtype=torch.float64, device="cuda")
    th = torch.zeros(4 * w.n, dtype=torch.float64, device="cuda")
    rc, infos = ctx.fit_batch(dw.design, dw.y, taus2, lams, dw.omega, w.block_ptr(), beta, z, th,
                              opts=dict(tol=1e-6, max_iter=cap, warm=3, warm_params=params.data_ptr()))
    bb, zz, tt = to_np(beta).reshape(4, -1), to_np(z).reshape(4, -1), to_np(th).reshape(4, -1)
    done = 0
    for ti, tau in enumerate(taus2):
        for li in range(2):
            f = ti * 2 + li
            if infos[f].status != 0:
                continue
            done += 1
            lam = lams[ti, li] * w.omega
            assert O.kkt(d.Xt, w.y, tau, lam, lmaxs[ti], bb[f], zz[f], tt[f]).value <= 1.001e-6
    assert done >= 1
