"""GPU parity of DLSC relaxation on K0 (Sec. 3.3.2, Alg. 2 with Mu = the
diagonal of the P2 velocity mass matrix on the high-order grid) and of the
DLSC-AMG preconditioner that relaxes with DLSC on every level (Sec. 4.1),
against the FP64 oracle, through the C ABI: one level-0 DLSC relaxation and
the FP64 cycle to 1e-12 (worst element and 2-norm), FP64 FGMRES within one
iteration of the oracle's, the FP32-preconditioned solve within two
iterations of the FP64 one, on C1 and at C2's full size."""
import numpy as np
import pytest

from oracle import direct, krylov
from problems import configs, mesh as M, stokes
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
def c1():
    return configs.c1()


def test_dlsc_level0_relaxation_fp64(sd, c1):
    prm = configs.th2d_dlsc(c1.nlevels)
    h = sd.stokes_setup(c1, dict(prm, precision=sd.STOKES_FP64))
    sd.stokes_factor_patches(h)
    o = make_oracle(c1, prm)
    rng = np.random.default_rng(41)
    n = c1.K[0].shape[0]
    x, b = rng.standard_normal(n), rng.standard_normal(n)
    y = torch.empty(n, dtype=torch.float64, device="cuda")
    sd.stokes_level_op(h, sd.STOKES_OP_RELAX, 0, dev(x), dev(b), y)
    assert rel(host(y), o.dl[0].sweep(x, b)) < 1e-12


def test_dlsc_level0_needs_the_mass_diagonal(sd, c1):
    import copy
    pr = copy.copy(c1)
    pr.Mu_diag = None
    with pytest.raises(sd.StokesError) as ei:
        sd.stokes_setup(pr, dict(configs.th2d_dlsc(pr.nlevels), precision=sd.STOKES_FP64))
    assert ei.value.code == sd.STOKES_ERR_INVALID_ARG


def test_dlsc_amg_cycle_and_solves_c1(sd, c1):
    prm = configs.th2d_dlsc(c1.nlevels)
    o = make_oracle(c1, prm)
    h64 = sd.stokes_setup(c1, dict(prm, precision=sd.STOKES_FP64))
    sd.stokes_factor_patches(h64)
    rng = np.random.default_rng(42)
    for r in (c1.b, rng.standard_normal(c1.b.size)):
        z = torch.empty(r.size, dtype=torch.float64, device="cuda")
        sd.stokes_vcycle(h64, dev(r), z)
        assert rel(host(z), o.apply(r)) < 1e-12
    xo, its_o, _ = krylov.fgmres(c1.K[0], c1.b, o.apply, rtol=1e-8, restart=30, maxit=200)
    its = {}
    sol = {}
    h32 = sd.stokes_setup(c1, dict(prm, precision=sd.STOKES_FP32))
    sd.stokes_factor_patches(h32)
    for prec, h in ((sd.STOKES_FP64, h64), (sd.STOKES_FP32, h32)):
        x = torch.zeros(c1.b.size, dtype=torch.float64, device="cuda")
        rc, info = sd.stokes_fgmres_solve(h, dev(c1.b), x, rtol=1e-8, restart=30, maxit=200)
        assert rc == sd.STOKES_OK and info[0][2] <= 1e-8
        its[prec] = info[0][0]
        sol[prec] = direct.zero_mean_pressure(host(x), c1.field_off[0], 2, c1.Mp)
    assert abs(its[sd.STOKES_FP64] - its_o) <= 1
    assert abs(its[sd.STOKES_FP32] - its[sd.STOKES_FP64]) <= 2
    xoz = direct.zero_mean_pressure(xo, c1.field_off[0], 2, c1.Mp)
    assert rel(sol[sd.STOKES_FP32], xoz) < 1e-5


def test_dlsc_amg_c2_full_size(sd):
    """The 256^2 problem with DLSC on every level: the FP64 cycle equals the
    oracle's on one application; FP32 reaches 1e-8 within +-2 iterations of
    the FP64 form."""
    pr = configs.c2()
    prm = configs.th2d_dlsc(pr.nlevels)
    h64 = sd.stokes_setup(pr, dict(prm, precision=sd.STOKES_FP64))
    sd.stokes_factor_patches(h64)
    o = make_oracle(pr, prm)
    r = np.random.default_rng(43).standard_normal(pr.b.size)
    z = torch.empty(r.size, dtype=torch.float64, device="cuda")
    sd.stokes_vcycle(h64, dev(r), z)
    assert rel(host(z), o.apply(r)) < 1e-12
    its = {}
    h32 = sd.stokes_setup(pr, dict(prm, precision=sd.STOKES_FP32))
    sd.stokes_factor_patches(h32)
    for prec, h in ((sd.STOKES_FP64, h64), (sd.STOKES_FP32, h32)):
        x = torch.zeros(pr.b.size, dtype=torch.float64, device="cuda")
        rc, info = sd.stokes_fgmres_solve(h, dev(pr.b), x, rtol=1e-8, restart=30, maxit=400)
        assert rc == sd.STOKES_OK and info[0][2] <= 1e-8
        its[prec] = info[0][0]
    assert abs(its[sd.STOKES_FP32] - its[sd.STOKES_FP64]) <= 2


def test_dlsc_batched_instances_fp64(sd):
    """Two Taylor-Hood instances in one handle (the same operator, so the
    same Chebyshev bounds, which batched DLSC requires; different right-hand
    sides), DLSC on every level: a batched handle keeps the level-sized DLSC
    operators with row masks (one-instance handles take the row-range
    sweep), and each instance's part of the FP64 cycle equals the oracle's."""
    probs = [stokes.build_th(M.unit_square(16), bc="noslip", rhs="random_b", seed=s) for s in (91, 92)]
    prm = configs.th2d_dlsc(probs[0].nlevels)
    h = sd.stokes_setup(probs, dict(prm, precision=sd.STOKES_FP64))
    sd.stokes_factor_patches(h)
    r = np.concatenate([np.random.default_rng(k).standard_normal(p.b.size) for k, p in enumerate(probs)])
    z = torch.empty(r.size, dtype=torch.float64, device="cuda")
    sd.stokes_vcycle(h, dev(r), z)
    zh = host(z)
    o = 0
    for p in probs:
        n = p.b.size
        assert rel(zh[o:o + n], make_oracle(p, prm).apply(r[o:o + n])) < 1e-12
        o += n
    sd.stokes_destroy(h)
