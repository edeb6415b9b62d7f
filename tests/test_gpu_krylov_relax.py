"""GPU parity of the Krylov-wrapped relaxation (Sec. 3.3.1: nu steps of
flexible GMRES per relaxation, each preconditioned by one undamped Vanka
sweep) against the FP64 oracle's `krylov_relax`: one relaxation per level
and whole cycles to 1e-12 in FP64, per-instance scalars in a batch, and the
FP32 FGMRES iteration count within +-2 of the FP64 one."""
import numpy as np
import pytest

from oracle import cycle, krylov
from problems import configs
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


def kprm(nlevels, nu=2, eta=1.0):
    return dict(schedule=0, nu1=nu, nu2=nu, eta_u=eta, eta_p=eta, omega=1.0,
                relax=[cycle.VANKA_KRYLOV] * (nlevels - 1))


@pytest.fixture(scope="module")
def c1():
    return configs.c1()


def test_krylov_relax_level_op_fp64(sd, c1):
    prm = kprm(c1.nlevels)
    h = sd.stokes_setup(c1, dict(prm, precision=sd.STOKES_FP64))
    assert sd.stokes_factor_patches(h) == 0
    o = make_oracle(c1, prm)
    rng = np.random.default_rng(21)
    for l in range(c1.nlevels - 1):
        n = c1.K[l].shape[0]
        x = rng.standard_normal(n)
        b = rng.standard_normal(n)
        y = torch.empty(n, dtype=torch.float64, device="cuda")
        sd.stokes_level_op(h, sd.STOKES_OP_RELAX, l, dev(x), dev(b), y)
        want = cycle.krylov_relax(o.K[l], x, b, o.vanka[l].apply, 2)
        assert rel(host(y), want) < 1e-12, l
    sd.stokes_destroy(h)


@pytest.mark.parametrize("nu", [1, 2, 3])
def test_krylov_cycle_fp64_matches_oracle(sd, c1, nu):
    prm = kprm(c1.nlevels, nu=nu, eta=0.75)
    h = sd.stokes_setup(c1, dict(prm, precision=sd.STOKES_FP64))
    assert sd.stokes_factor_patches(h) == 0
    o = make_oracle(c1, prm)
    rng = np.random.default_rng(22 + nu)
    n = c1.K[0].shape[0]
    for _ in range(2):
        r = rng.standard_normal(n)
        z = torch.empty(n, dtype=torch.float64, device="cuda")
        sd.stokes_vcycle(h, dev(r), z)
        assert rel(host(z), o.apply(r)) < 1e-12
    sd.stokes_destroy(h)


def test_krylov_relax_batched_instances_keep_their_own_scalars(sd):
    """Two instances of different sizes in one handle give, each, the cycle
    of its own single-instance handle (per-instance Krylov scalars)."""
    pa, pb = configs.c2(16), configs.c2(24)
    prm_a, prm_b = kprm(pa.nlevels), kprm(pb.nlevels)
    hb = sd.stokes_setup([pa, pb], dict(prm_a if pa.nlevels >= pb.nlevels else prm_b, precision=sd.STOKES_FP64))
    assert sd.stokes_factor_patches(hb) == 0
    na, nb = pa.K[0].shape[0], pb.K[0].shape[0]
    rng = np.random.default_rng(30)
    ra, rb = rng.standard_normal(na), rng.standard_normal(nb)
    z = torch.empty(na + nb, dtype=torch.float64, device="cuda")
    sd.stokes_vcycle(hb, dev(np.concatenate([ra, rb])), z)
    zz = host(z)
    for pr, p1, r, part in ((pa, prm_a, ra, zz[:na]), (pb, prm_b, rb, zz[na:])):
        o = make_oracle(pr, p1)
        assert rel(part, o.apply(r)) < 1e-12
    sd.stokes_destroy(hb)


def test_krylov_fgmres_fp32_within_two_iterations(sd):
    pr = configs.c2(48)
    prm = kprm(pr.nlevels)
    its = {}
    for prec in (sd.STOKES_FP64, sd.STOKES_FP32):
        h = sd.stokes_setup(pr, dict(prm, precision=prec))
        assert sd.stokes_factor_patches(h) == 0
        n = pr.K[0].shape[0]
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        st, info = sd.stokes_fgmres_solve(h, dev(pr.b), x, 1e-8, 30, 200)
        iters, status, relres = info[0]
        assert st == 0 and status == 0 and relres <= 1e-8
        its[prec] = iters
        sd.stokes_destroy(h)
    o = make_oracle(pr, prm)
    _, oits, orel = krylov.fgmres(pr.K[0], pr.b, o.apply, rtol=1e-8, restart=30, maxit=200)
    assert orel <= 1e-8
    assert abs(its[sd.STOKES_FP64] - oits) <= 1
    assert abs(its[sd.STOKES_FP32] - oits) <= 2
