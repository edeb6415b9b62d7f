"""GPU parity in 3D (Taylor-Hood on Kuhn tetrahedra, 196-DoF patches,
coarse patches through the global-memory factor and apply paths) and for
batched instances, against the FP64 oracle through the C ABI; the full
32^3 cavity is checked on sampled Vanka entries and by solve properties."""
import numpy as np
import pytest

from oracle import krylov, vanka
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
def cube():
    return stokes.build_th(M.unit_cube(4), bc="lid")


@pytest.mark.parametrize("relax", ["vanka", "dlsc"])
def test_3d_cycle_fp64_matches_oracle(sd, cube, relax):
    prm = dict(configs.TH3D_VANKA, cheb_deg=(4, 4, 16))
    if relax == "dlsc":
        prm["relax"] = [0] + [1] * (cube.nlevels - 2)
    h = sd.stokes_setup(cube, dict(prm, precision=sd.STOKES_FP64))
    sd.stokes_factor_patches(h)
    o = make_oracle(cube, prm)
    r = np.random.default_rng(31).standard_normal(cube.b.size)
    z = torch.empty(r.size, dtype=torch.float64, device="cuda")
    sd.stokes_vcycle(h, dev(r), z)
    assert rel(host(z), o.apply(r)) < 1e-12


def test_3d_large_coarse_patches_fp64(sd):
    """A 8^3 cavity has coarse patches of several hundred DoFs (global-memory
    factorisation and apply)."""
    pr = stokes.build_th(M.unit_cube(8), bc="lid")
    assert max(np.diff(p.ptr).max() for p in pr.patches) > 300
    prm = dict(configs.TH3D_VANKA)
    h = sd.stokes_setup(pr, dict(prm, precision=sd.STOKES_FP64))
    sd.stokes_factor_patches(h)
    o = make_oracle(pr, prm)
    r = np.random.default_rng(32).standard_normal(pr.b.size)
    z = torch.empty(r.size, dtype=torch.float64, device="cuda")
    sd.stokes_vcycle(h, dev(r), z)
    assert rel(host(z), o.apply(r)) < 1e-12


@pytest.mark.parametrize("tcgen05", [0, 1])
def test_3d_large_coarse_patches_fp32(sd, tcgen05):
    """FP32 on the 8^3 cavity: patches with m > 32 velocity DoFs per
    component are factorised by the blocked sweep on tensor cores (3xTF32;
    with tcgen05 = 1 the three-tile-row blocks run their trailing products as
    tcgen05.mma with TMEM accumulators) and those outside the bulk-copy bins
    are solved from tiled blocks; every level's Vanka op agrees with the FP64
    oracle to FP32 accuracy, and the FP32 cycle with the FP64 oracle cycle to
    1e-5."""
    pr = stokes.build_th(M.unit_cube(8), bc="lid")
    prm = dict(configs.TH3D_VANKA, factor_tcgen05=tcgen05)
    assert max(int(np.asarray(p.nvel)[:, 0].max()) for p in pr.patches[:2]) == 65  # three tile rows
    h = sd.stokes_setup(pr, dict(prm, precision=sd.STOKES_FP32))
    assert sd.stokes_factor_patches(h) == 0
    o = make_oracle(pr, prm)
    rng = np.random.default_rng(35)
    for l in range(pr.nlevels - 1):
        m = np.asarray(pr.patches[l].nvel)[:, 0]
        n = pr.K[l].shape[0]
        x = rng.standard_normal(n)
        y = torch.empty(n, dtype=torch.float64, device="cuda")
        sd.stokes_level_op(h, sd.STOKES_OP_VANKA, l, dev(x), None, y)
        assert rel(host(y), o.vanka[l].apply(x)) < 2e-5, (l, int(m.max()))
    assert max(int(np.asarray(p.nvel)[:, 0].max()) for p in pr.patches) > 96
    r = rng.standard_normal(pr.b.size)
    z = torch.empty(r.size, dtype=torch.float64, device="cuda")
    sd.stokes_vcycle(h, dev(r), z)
    assert rel(host(z), o.apply(r)) < 1e-5


def test_3d_fgmres_fp32_within_two_iterations(sd, cube):
    prm = dict(configs.TH3D_VANKA)
    o = make_oracle(cube, prm)
    _, its_o, _ = krylov.fgmres(cube.K[0], cube.b, o.apply, rtol=1e-8, restart=30, maxit=200)
    h = sd.stokes_setup(cube, dict(prm, precision=sd.STOKES_FP32))
    sd.stokes_factor_patches(h)
    x = torch.zeros(cube.b.size, dtype=torch.float64, device="cuda")
    rc, info = sd.stokes_fgmres_solve(h, dev(cube.b), x, rtol=1e-8, restart=30, maxit=200)
    assert rc == sd.STOKES_OK and info[0][2] <= 1e-8
    assert abs(info[0][0] - its_o) <= 2


@pytest.fixture(scope="module")
def c4():
    return configs.c4()


def test_c4_full_size_sampled_vanka_and_solve(sd, c4):
    prm = dict(configs.TH3D_VANKA)
    h64 = sd.stokes_setup(c4, dict(prm, precision=sd.STOKES_FP64))
    assert sd.stokes_factor_patches(h64) == 0
    rng = np.random.default_rng(33)
    for l in (0, 1, 2):
        n = c4.K[l].shape[0]
        r = rng.standard_normal(n)
        y = torch.empty(n, dtype=torch.float64, device="cuda")
        sd.stokes_level_op(h64, sd.STOKES_OP_VANKA, l, dev(r), None, y)
        covered = np.nonzero(np.bincount(c4.patches[l].dof, minlength=n))[0]
        dofs = rng.choice(covered, size=40, replace=False)
        ref = vanka.sampled_apply(c4.K[l], c4.patches[l], r, dofs)
        assert rel(host(y)[dofs], ref) < 1e-11, l
    # the coarsest relaxed level (a few hundred large patches) in full
    lc = c4.nlevels - 2
    n = c4.K[lc].shape[0]
    r = rng.standard_normal(n)
    y = torch.empty(n, dtype=torch.float64, device="cuda")
    sd.stokes_level_op(h64, sd.STOKES_OP_VANKA, lc, dev(r), None, y)
    assert rel(host(y), vanka.VankaLevel(c4.K[lc], c4.patches[lc]).apply(r)) < 1e-11
    # FP32 and FP64 preconditioned solves reach 1e-8 within +-2 iterations
    b = dev(c4.b)
    its = {}
    xs = {}
    for prec in (sd.STOKES_FP64, sd.STOKES_FP32):
        h = h64 if prec == sd.STOKES_FP64 else sd.stokes_setup(c4, dict(prm, precision=prec))
        if prec == sd.STOKES_FP32:
            sd.stokes_factor_patches(h)
        x = torch.zeros_like(b)
        rc, info = sd.stokes_fgmres_solve(h, b, x, rtol=1e-8, restart=30, maxit=400)
        assert rc == sd.STOKES_OK and info[0][2] <= 1e-8
        its[prec] = info[0][0]
        xs[prec] = host(x)
    assert abs(its[sd.STOKES_FP32] - its[sd.STOKES_FP64]) <= 2
    assert rel(xs[sd.STOKES_FP32], xs[sd.STOKES_FP64]) < 1e-5


def test_batched_small_c5_like_matches_oracle(sd):
    inst = configs.c5_instances(count=6, lo=6, hi=20, seed=777)
    probs = [stokes.build_th(M.unit_square(n), nu=nu, bc="noslip", rhs="random_b", seed=s) for n, nu, s in inst]
    prm = dict(configs.TH2D_VANKA)
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


def test_c5_full_batch_solves_every_instance(sd):
    """64 instances (n ~ U{32..192}, nu ~ 10^U(-2,2)) in one handle: every
    instance reaches the 1e-8 true residual with its own FGMRES scalars, and
    the smallest instance's cycle equals the oracle's."""
    probs = configs.c5()
    prm = dict(configs.TH2D_VANKA)
    h = sd.stokes_setup(probs, dict(prm, precision=sd.STOKES_FP32))
    sd.stokes_factor_patches(h)
    b = np.concatenate([p.b for p in probs])
    x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
    rc, info = sd.stokes_fgmres_solve(h, dev(b), x, rtol=1e-8, restart=30, maxit=600)
    assert rc == sd.STOKES_OK
    xh = host(x)
    o = 0
    for k, p in enumerate(probs):
        n = p.b.size
        assert info[k][2] <= 1e-8
        assert np.linalg.norm(p.b - p.K[0] @ xh[o:o + n]) <= 1.01e-8 * np.linalg.norm(p.b)
        o += n
    # FP64 cycle of the whole batch against the oracle on the smallest, the
    # largest, the shallowest and the deepest instance
    h64 = sd.stokes_setup(probs, dict(prm, precision=sd.STOKES_FP64))
    sd.stokes_factor_patches(h64)
    r = np.random.default_rng(34).standard_normal(b.size)
    z = torch.empty(b.size, dtype=torch.float64, device="cuda")
    sd.stokes_vcycle(h64, dev(r), z)
    zh = host(z)
    sizes = [p.b.size for p in probs]
    depth = [p.nlevels for p in probs]
    picks = {int(np.argmin(sizes)), int(np.argmax(sizes)), int(np.argmin(depth)), int(np.argmax(depth))}
    assert min(depth) < max(depth)
    for k in sorted(picks):
        o = sum(sizes[:k])
        n = sizes[k]
        assert rel(zh[o:o + n], make_oracle(probs[k], prm).apply(r[o:o + n])) < 1e-12, k
    # the smallest instance's FP32-preconditioned solution against the oracle's
    from oracle import direct
    k = int(np.argmin(sizes))
    p = probs[k]
    o = sum(sizes[:k])
    xo, _, _ = krylov.fgmres(p.K[0], p.b, make_oracle(p, prm).apply, rtol=1e-8, restart=30, maxit=600)
    off = p.field_off[0]
    assert rel(direct.zero_mean_pressure(xh[o:o + sizes[k]], off, 2, p.Mp),
               direct.zero_mean_pressure(xo, off, 2, p.Mp)) < 1e-5
