"""GPU parity for Scott-Vogelius P2/P1disc (3-seed cell patches, the
L2-projection pressure restriction) and for DLSC relaxation, against the
FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from oracle import krylov
from problems import configs, stokes
from tests.helpers import make_oracle, rel

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


@pytest.fixture(scope="module")
def sv16():
    return stokes.build_sv(16)


def variants(pr):
    return {"vanka": dict(configs.SV2D_VANKA), "vanka-dlsc": configs.sv_vanka_dlsc(pr.nlevels)}


@pytest.mark.parametrize("name", ["vanka", "vanka-dlsc"])
def test_sv_cycle_fp64_matches_oracle(sd, sv16, name):
    prm = variants(sv16)[name]
    h = sd.stokes_setup(sv16, dict(prm, precision=sd.STOKES_FP64))
    sd.stokes_factor_patches(h)
    o = make_oracle(sv16, prm)
    rng = np.random.default_rng(21)
    for r in (sv16.b, rng.standard_normal(sv16.b.size)):
        z = torch.empty(r.size, dtype=torch.float64, device="cuda")
        sd.stokes_vcycle(h, dev(r), z)
        assert rel(host(z), o.apply(r)) < 1e-12


def test_sv_level_ops_fp64(sd, sv16):
    prm = variants(sv16)["vanka-dlsc"]
    h = sd.stokes_setup(sv16, dict(prm, precision=sd.STOKES_FP64))
    sd.stokes_factor_patches(h)
    o = make_oracle(sv16, prm)
    rng = np.random.default_rng(22)
    # level 0: three-seed Vanka
    n0 = sv16.K[0].shape[0]
    x = rng.standard_normal(n0)
    y = torch.empty(n0, dtype=torch.float64, device="cuda")
    sd.stokes_level_op(h, sd.STOKES_OP_VANKA, 0, dev(x), None, y)
    assert rel(host(y), o.vanka[0].apply(x)) < 1e-12
    # level 1: one DLSC relaxation call (two sweeps)
    n1 = sv16.K[1].shape[0]
    x1 = rng.standard_normal(n1)
    b1 = rng.standard_normal(n1)
    y1 = torch.empty(n1, dtype=torch.float64, device="cuda")
    sd.stokes_level_op(h, sd.STOKES_OP_RELAX, 1, dev(x1), dev(b1), y1)
    assert rel(host(y1), o.dl[1].sweep(x1, b1)) < 1e-12


@pytest.mark.parametrize("name", ["vanka", "vanka-dlsc"])
def test_sv_fgmres_fp32(sd, sv16, name):
    prm = variants(sv16)[name]
    o = make_oracle(sv16, prm)
    _, its_o, _ = krylov.fgmres(sv16.K[0], sv16.b, o.apply, rtol=1e-8, restart=30, maxit=300)
    h = sd.stokes_setup(sv16, dict(prm, precision=sd.STOKES_FP32))
    sd.stokes_factor_patches(h)
    x = torch.zeros(sv16.b.size, dtype=torch.float64, device="cuda")
    rc, info = sd.stokes_fgmres_solve(h, dev(sv16.b), x, rtol=1e-8, restart=30, maxit=300)
    assert rc == sd.STOKES_OK and info[0][2] <= 1e-8
    assert abs(info[0][0] - its_o) <= 2
    xh = host(x)
    # the converged velocity is divergence-free to the accuracy of the solve
    off = sv16.field_off[0]
    A = sv16.K[0][: off[2], : off[2]]
    energy = np.sqrt(xh[: off[2]] @ (A @ xh[: off[2]]))
    assert stokes.divergence_norm(sv16, xh) < 1e-6 * energy


def test_th_dlsc_on_coarse_levels_fp64(sd):
    pr = configs.c1()
    prm = dict(configs.TH2D_VANKA, relax=[0] + [1] * (pr.nlevels - 2))
    h = sd.stokes_setup(pr, dict(prm, precision=sd.STOKES_FP64))
    sd.stokes_factor_patches(h)
    o = make_oracle(pr, prm)
    r = np.random.default_rng(23).standard_normal(pr.b.size)
    z = torch.empty(r.size, dtype=torch.float64, device="cuda")
    sd.stokes_vcycle(h, dev(r), z)
    assert rel(host(z), o.apply(r)) < 1e-12


@pytest.fixture(scope="module")
def c3():
    return configs.c3()


@pytest.mark.parametrize("name", ["vanka", "vanka-dlsc"])
def test_c3_full_size(sd, c3, name):
    """The 128^2 Alfeld problem: the FP64 cycle equals the oracle's on one
    application; the FP32-preconditioned solve reaches 1e-8 within +-2
    iterations of the FP64 form and a divergence-free velocity."""
    prm = variants(c3)[name]
    h64 = sd.stokes_setup(c3, dict(prm, precision=sd.STOKES_FP64))
    sd.stokes_factor_patches(h64)
    o = make_oracle(c3, prm)
    r = np.random.default_rng(24).standard_normal(c3.b.size)
    z = torch.empty(r.size, dtype=torch.float64, device="cuda")
    sd.stokes_vcycle(h64, dev(r), z)
    assert rel(host(z), o.apply(r)) < 1e-12
    its = {}
    for prec, h in ((sd.STOKES_FP64, h64), (sd.STOKES_FP32, None)):
        if h is None:
            h = sd.stokes_setup(c3, dict(prm, precision=prec))
            sd.stokes_factor_patches(h)
        x = torch.zeros(c3.b.size, dtype=torch.float64, device="cuda")
        rc, info = sd.stokes_fgmres_solve(h, dev(c3.b), x, rtol=1e-8, restart=30, maxit=400)
        assert rc == sd.STOKES_OK and info[0][2] <= 1e-8
        its[prec] = info[0][0]
        xh = host(x)
    assert abs(its[sd.STOKES_FP32] - its[sd.STOKES_FP64]) <= 2
    off = c3.field_off[0]
    A = c3.K[0][: off[2], : off[2]]
    energy = np.sqrt(xh[: off[2]] @ (A @ xh[: off[2]]))
    assert stokes.divergence_norm(c3, xh) < 1e-6 * energy
