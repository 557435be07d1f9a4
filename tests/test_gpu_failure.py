"""Failure detection on the GPU without a GPU fault: a bounded device wait
that nothing completes runs out, records its code and returns, the call ends
with FSQR_ETIMEOUT, and the context keeps working (a wait that is completed
succeeds). The host-side failures (invalid arguments, NaN inputs, max_iter,
the wall-clock timeout) are covered in the parity and edge-case tests.
"""
import time

import pytest

from paper_2601_02826_gb300 import synth

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


def test_a_wait_that_nothing_completes_runs_out_and_reports(ctx):
    from paper_2601_02826_gb300 import fsqr
    t0 = time.perf_counter()
    rc, ok = ctx.wait_selftest(2_000_000, arrive=False)  # about a millisecond
    assert rc == fsqr.ETIMEOUT and ok == 0
    assert "budget" in ctx.last_error()
    assert time.perf_counter() - t0 < 30
    rc, ok = ctx.wait_selftest(2_000_000, arrive=True)
    assert rc == fsqr.OK and ok == 1


def test_context_is_usable_after_an_expired_wait(ctx):
    from paper_2601_02826_gb300.device import upload
    ctx.wait_selftest(1000, arrive=False)
    w = synth.tiny_geno(701, 120, 90, c=0, fmt=1, G=2, taus=(0.5,))
    dw = upload(ctx, w)
    assert ctx.lambda_max(dw.design, dw.y, 0.5, dw.omega) > 0
