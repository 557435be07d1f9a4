"""Fits of the 10,000 x 500,000 int8 grid workload (ragged blocks U(5k, 30k))
solved to KKT <= 1e-6 on the GPU in the bench's configuration: wide slot
groups (32 slots), tensor-core passes, and the oracle's stop test on the full
design for sampled fits, formed one block of 20,000 columns at a time (the
dense FP64 design would take 40 GB). The fits are the small-lambda end of the
9 tau x 20 lambda grid (lambda = 0.0127 and 0.01 lambda_max), which converge
within a few 10^5 steps; the fits near lambda_max need more than 10^6 (see the
design notes), so the whole grid is not a test.

It runs for several minutes, so it is opt-in: FSQR_LONG_TESTS=1.
"""
import os
import time

import numpy as np
import pytest

from oracle import fsqrppa as O
from paper_2601_02826_gb300 import synth
from tests.gpu_helpers import to_np

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(os.environ.get("FSQR_LONG_TESTS") != "1", reason="long test: FSQR_LONG_TESTS=1")]


def _oracle_kkt_blockwise(w, fits, chunk=20_000):
    """Oracle KKT of (tau, lam_vec, lam_norm, beta, z, theta) fits on the
    standardised grid design, one block of stored columns at a time."""
    n, P = w.n, w.P
    xb = [np.full(n, f["beta"][0]) for f in fits]          # intercept column
    s = [np.zeros(P) for _ in fits]
    for k, f in enumerate(fits):
        s[k][0] = float(np.sum(f["theta"]))
    g = O.decode_stored(w.geno, w.fmt, n)
    for j0 in range(0, w.p, chunk):
        j1 = min(w.p, j0 + chunk)
        Xc = O.build_design(g[j0:j1], np.zeros((0, n))).Xt[:, 1:]
        for k, f in enumerate(fits):
            s[k][1 + j0:1 + j1] = Xc.T @ f["theta"]
            bc = f["beta"][1 + j0:1 + j1]
            nz = np.flatnonzero(bc)
            if nz.size:
                xb[k] += Xc[:, nz] @ bc[nz]
    return [O.kkt_from_products(w.y, f["tau"], f["lam"], f["lam_norm"], f["beta"], f["z"], f["theta"], xb[k], s[k])
            for k, f in enumerate(fits)]


def test_grid_fits_converge_and_meet_the_oracle_stop_test():
    from paper_2601_02826_gb300 import fsqr
    from paper_2601_02826_gb300.device import upload
    torch.cuda.set_device(0)
    ctx = fsqr.Context(0, torch.cuda.current_stream().cuda_stream)
    w = synth.grid_int8()
    dw = upload(ctx, w)
    taus = w.taus
    fr = np.asarray(w.lambda_fracs)[-2:]
    lm = [ctx.lambda_max(dw.design, dw.y, t, dw.omega) for t in taus]
    lam = np.array([[f * l for f in fr] for l in lm])
    B = lam.size
    beta = torch.zeros(B * w.P, dtype=torch.float64, device="cuda")
    z = torch.zeros(B * w.n, dtype=torch.float64, device="cuda")
    th = torch.zeros(B * w.n, dtype=torch.float64, device="cuda")
    ctx.profile(reset=True)
    t0 = time.time()
    rc, infos = ctx.fit_batch(dw.design, dw.y, taus, lam, dw.omega, w.block_ptr(), beta, z, th,
                              opts=dict(tol=1e-6, max_iter=800_000, precision=fsqr.MIXED, max_group=32,
                                        timeout_ms=1_200_000))
    wall = time.time() - t0
    prof = ctx.profile()
    print(f"grid fits: rc={rc} wall={wall:.1f}s fits/s={B / wall:.4f} steps={prof.iterations} "
          f"iters={[i.iters for i in infos]} kkt={[round(i.kkt, 9) for i in infos]}")
    assert all(i.status == 0 for i in infos), [i.status for i in infos]
    bb, zz, tt = to_np(beta).reshape(B, -1), to_np(z).reshape(B, -1), to_np(th).reshape(B, -1)
    picks = [(0, 1), (4, 0), (8, 1)]
    fits = []
    for t, l in picks:
        f = t * len(fr) + l
        fits.append(dict(tau=taus[t], lam=lam[t, l] * w.omega, lam_norm=lm[t], beta=bb[f], z=zz[f], theta=tt[f]))
    for (t, l), ko in zip(picks, _oracle_kkt_blockwise(w, fits)):
        assert ko.value <= 1.001e-6, (t, l, ko)
    ctx.close()
