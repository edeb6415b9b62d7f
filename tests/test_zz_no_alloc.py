"""The no-allocation Vanka entry point (stokes_vanka_noalloc) against the
regular one (stokes_level_op, STOKES_OP_VANKA), through the C ABI.

Callers that cannot allocate device memory while they run (a fixed memory
budget, or a context where cudaMalloc is not permitted) use the variant
whose scratch is a fixed array inside the library.  It runs the same kernels
in the same order on the same data as the regular entry point, only with
another scratch, so two calls in a row must each give the regular result bit
for bit; the second call also shows that the contents left in the shared
scratch by the first do not leak into a result.  A pipeline error flag that
is set (as a bulk-copy wait that ran out would set it) must make the call
fail.  This file is collected last on purpose."""
import numpy as np
import pytest

from problems import configs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_vanka_matches_regular_entry_point(precision):
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2306_06795_gb300 as sd

    prec = sd.STOKES_FP64 if precision == "fp64" else sd.STOKES_FP32
    pr = configs.c1()
    h = sd.stokes_setup(pr, dict(configs.TH2D_VANKA, precision=prec))
    sd.stokes_factor_patches(h)
    rng = np.random.default_rng(99)
    for level in (0, 1):
        n = pr.K[level].shape[0]
        for call in range(2):
            x = torch.tensor(rng.standard_normal(n), dtype=torch.float64, device="cuda")
            y_ref = torch.empty_like(x)
            y_new = torch.full_like(x, float("nan"))
            sd.stokes_level_op(h, sd.STOKES_OP_VANKA, level, x, None, y_ref)
            sd.stokes_vanka_noalloc(h, level, x, y_new)
            torch.cuda.synchronize()
            assert torch.isfinite(y_new).all(), (level, call)
            assert torch.equal(y_new, y_ref), (level, call, float((y_new - y_ref).abs().max()))


def test_noalloc_rejects_levels_beyond_its_scratch():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2306_06795_gb300 as sd

    # C2 level 0 in FP64 needs 2 x 4.7 MB + 20.4 MB < 32 MiB; a batch of
    # two C2 problems needs more than the fixed scratch
    pr = configs.c2()
    h = sd.stokes_setup([pr, pr], dict(configs.TH2D_VANKA, precision=sd.STOKES_FP64))
    sd.stokes_factor_patches(h)
    n = 2 * pr.K[0].shape[0]
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(sd.StokesError) as ei:
        sd.stokes_vanka_noalloc(h, 0, x, torch.empty_like(x))
    assert ei.value.code == sd.STOKES_ERR_INVALID_ARG


def test_noalloc_reports_a_pipeline_error_flag():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2306_06795_gb300 as sd

    pr = configs.c1()
    h = sd.stokes_setup(pr, dict(configs.TH2D_VANKA, precision=sd.STOKES_FP32))
    sd.stokes_factor_patches(h)
    n = pr.K[0].shape[0]
    x = torch.ones(n, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    sd.stokes_vanka_noalloc(h, 0, x, y)  # clean flags: accepted
    sd.stokes_inject_pipeline_error(h, 0)
    with pytest.raises(sd.StokesError) as ei:
        sd.stokes_vanka_noalloc(h, 0, x, y)
    assert ei.value.code == sd.STOKES_ERR_CUDA
    # the regular entry point reads the same flags
    with pytest.raises(sd.StokesError) as ei:
        sd.stokes_level_op(h, sd.STOKES_OP_VANKA, 0, x, None, y)
    assert ei.value.code == sd.STOKES_ERR_CUDA
