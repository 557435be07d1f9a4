"""fsqr_lambda_max_noalloc against fsqr_lambda_max.

The variant runs the same kernels on buffers carved from a static device
array instead of the context's workspace. Its results must equal those of
the workspace entry point. The array keeps the previous call's bytes, so each
case is called twice in a row, and the cases alternate in size. The file
name sorts last, so in a full run these tests also follow every other GPU
test in the same process. They pass when run alone in a fresh process too.
"""
import numpy as np
import pytest

from oracle import fsqrppa as O
from paper_2601_02826_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    "int8": lambda: synth.tiny_geno(112, 333, 1000, c=2, fmt=synth.FMT_INT8, G=5, taus=(0.3,)),
    "dense": lambda: synth.small_dense(seed=101, n=61, p=150, G=3, tau=0.5),
    "rows": lambda: synth.tiny_geno(104, 2500, 300, c=1, fmt=synth.FMT_INT8, G=2, taus=(0.5,)),
    "2bit": lambda: synth.tiny_geno(103, 257, 700, c=0, fmt=synth.FMT_2BIT, G=4, taus=(0.7,)),
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


def test_noalloc_matches_workspace_entry_point(ctx):
    ups = {}
    for k, make in CASES.items():
        w = make()
        ups[k] = (w, _up(ctx, w))
    for case in ["int8", "dense", "rows", "2bit", "int8"]:
        w, dw = ups[case]
        for tau in (0.3, 0.8):
            first = ctx.lambda_max_noalloc(dw.design, dw.y, tau, dw.omega)
            second = ctx.lambda_max_noalloc(dw.design, dw.y, tau, dw.omega)
            ref = ctx.lambda_max(dw.design, dw.y, tau, dw.omega)
            assert first == pytest.approx(ref, rel=1e-12, abs=0.0), (case, tau, first, ref)
            assert second == pytest.approx(ref, rel=1e-12, abs=0.0), (case, tau, second, ref)
            d = O.build_design(O.decode_stored(w.geno, w.fmt, w.n), w.cov)
            assert first == pytest.approx(O.lambda_max(d.Xt, w.y, tau, w.omega), rel=1e-10)


def test_noalloc_allocates_no_device_memory(ctx):
    w = CASES["int8"]()
    dw = _up(ctx, w)
    ctx.lambda_max_noalloc(dw.design, dw.y, 0.5, dw.omega)  # first call: set-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    got = [ctx.lambda_max_noalloc(dw.design, dw.y, t, dw.omega) for t in (0.2, 0.6)]
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert all(np.isfinite(got)) and min(got) > 0.0


def test_noalloc_rejects_designs_beyond_the_static_scratch(ctx):
    from paper_2601_02826_gb300 import fsqr
    n, p = 16, 300_000  # about 40 bytes per column: 12 MB > 8 MiB
    geno = torch.zeros(p * 16, dtype=torch.uint8, device="cuda")
    y = torch.arange(n, dtype=torch.float64, device="cuda")
    omega = torch.ones(1 + p, dtype=torch.float64, device="cuda")
    omega[0] = 0.0
    d = ctx.design(n, p, 0, fsqr.INT8, geno, 16, standardize=1)
    with pytest.raises(fsqr.FsqrError) as e:
        ctx.lambda_max_noalloc(d, y, 0.5, omega)
    assert e.value.code == fsqr.EINVAL
    assert "FSQR_NOALLOC_SCRATCH_BYTES" in str(e.value)
    # the workspace entry point handles the same design
    assert ctx.lambda_max(d, y, 0.5, omega) >= 0.0
