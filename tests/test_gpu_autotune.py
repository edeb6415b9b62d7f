"""The Vanka-apply autotuner: it reports its per-bin choices as JSON, and
the cycle after tuning (new tiles, ring depth, grid; graphs recaptured) is
bitwise the cycle before it, in FP64 and FP32."""
import json

import numpy as np
import pytest

from problems import configs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sd():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2306_06795_gb300 as sd
    return sd


@pytest.mark.parametrize("prec", [0, 1])
def test_autotune_keeps_the_cycle_bitwise(sd, prec):
    pr = configs.c2(64)
    h = sd.stokes_setup(pr, dict(configs.TH2D_VANKA, precision=prec))
    assert sd.stokes_factor_patches(h) == 0
    n = pr.K[0].shape[0]
    r = torch.tensor(np.random.default_rng(50).standard_normal(n), device="cuda")
    z0 = torch.empty_like(r)
    z1 = torch.empty_like(r)
    sd.stokes_vcycle(h, r, z0)
    sd.stokes_autotune(h, 3)
    rep = json.loads(sd.stokes_autotune_report(h))
    assert rep["bins"], rep
    for b in rep["bins"]:
        assert b["tile_patches"] >= 4 and b["stages"] in (2, 3) and b["grid"] >= 1 and b["us"] > 0
    sd.stokes_vcycle(h, r, z1)
    torch.cuda.synchronize()
    assert torch.equal(z0, z1)
    sd.stokes_destroy(h)
