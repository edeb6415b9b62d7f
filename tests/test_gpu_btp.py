"""GPU parity of the block-triangular comparison preconditioner BTP (Sec. 4)
against the FP64 oracle: one application to 1e-12 in FP64 for Taylor-Hood
(SA V-cycles on A and on M_p / nu) and Scott-Vogelius (exact block-diagonal
mass inverse), and the FP32 FGMRES iteration count within +-2 of the FP64
oracle's."""
import numpy as np
import pytest

from oracle import btp as obtp, krylov
from problems import btp as pbtp, configs
from tests.helpers import rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sd():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2306_06795_gb300 as sd
    return sd


def dev(a):
    return torch.tensor(np.asarray(a, dtype=np.float64), device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def with_btp(pr):
    pr.btp = pbtp.build_btp(pr)
    return pr


PRM = dict(configs.TH2D_VANKA, preconditioner=1, btp_steps=2)


@pytest.mark.parametrize("which", ["th", "sv"])
def test_btp_application_fp64_matches_oracle(sd, which):
    pr = with_btp(configs.c1() if which == "th" else configs.c3(8))
    prm = dict(PRM) if which == "th" else dict(configs.SV2D_VANKA, preconditioner=1, btp_steps=2)
    h = sd.stokes_setup(pr, dict(prm, precision=sd.STOKES_FP64))
    o = obtp.BTPOracle(pr.btp, steps=2)
    rng = np.random.default_rng(40)
    n = pr.K[0].shape[0]
    for _ in range(2):
        r = rng.standard_normal(n)
        z = torch.empty(n, dtype=torch.float64, device="cuda")
        sd.stokes_vcycle(h, dev(r), z)
        assert rel(host(z), o.apply(r)) < 1e-12
    sd.stokes_destroy(h)


def test_btp_fgmres_fp32_within_two_iterations(sd):
    pr = with_btp(configs.c2(32))
    its = {}
    for prec in (sd.STOKES_FP64, sd.STOKES_FP32):
        h = sd.stokes_setup(pr, dict(PRM, precision=prec))
        n = pr.K[0].shape[0]
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        st, info = sd.stokes_fgmres_solve(h, dev(pr.b), x, 1e-8, 30, 400)
        iters, status, relres = info[0]
        assert st == 0 and status == 0 and relres <= 1e-8
        its[prec] = iters
        sd.stokes_destroy(h)
    o = obtp.BTPOracle(pr.btp, steps=2)
    _, oits, orel = krylov.fgmres(pr.K[0], pr.b, o.apply, rtol=1e-8, restart=30, maxit=400)
    assert orel <= 1e-8
    assert abs(its[sd.STOKES_FP64] - oits) <= 1
    assert abs(its[sd.STOKES_FP32] - oits) <= 2
