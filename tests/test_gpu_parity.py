"""GPU parity of the CUDA solve path against the FP64 oracle, through the
C ABI.  FP64 cycle: 1e-12 relative (the tolerance stated for the FP64
preconditioner); FP32 cycle: 1e-5 relative on one application (FP32
rounding of ~1e3-term sums, amplified by the cycle's norm), and FGMRES to
the same 1e-8 true residual within +-2 iterations of the FP64 form."""
import numpy as np
import pytest

from oracle import krylov
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


PRM = configs.TH2D_VANKA


@pytest.fixture(scope="module")
def c1():
    return configs.c1()


@pytest.fixture(scope="module")
def h64(sd, c1):
    h = sd.stokes_setup(c1, dict(PRM, precision=sd.STOKES_FP64))
    assert sd.stokes_factor_patches(h) == 0
    return h


@pytest.fixture(scope="module")
def h32(sd, c1):
    h = sd.stokes_setup(c1, dict(PRM, precision=sd.STOKES_FP32))
    assert sd.stokes_factor_patches(h) == 0
    return h


def test_level_ops_fp64(sd, c1, h64):
    o = make_oracle(c1, PRM)
    rng = np.random.default_rng(10)
    L = c1.nlevels
    assert sd.stokes_num_levels(h64) == L
    for l in range(L):
        n = c1.K[l].shape[0]
        assert sd.stokes_level_size(h64, l) == n
        x = rng.standard_normal(n)
        b = rng.standard_normal(n)
        y = torch.empty(n, dtype=torch.float64, device="cuda")
        for op in (sd.STOKES_OP_SPMV, sd.STOKES_OP_SPMV_F64):
            sd.stokes_level_op(h64, op, l, dev(x), None, y)
            assert rel(host(y), c1.K[l] @ x) < 1e-14
        sd.stokes_level_op(h64, sd.STOKES_OP_RESIDUAL, l, dev(x), dev(b), y)
        assert rel(host(y), b - c1.K[l] @ x) < 1e-14
        if l + 1 < L:
            nc = c1.K[l + 1].shape[0]
            yc = torch.empty(nc, dtype=torch.float64, device="cuda")
            sd.stokes_level_op(h64, sd.STOKES_OP_RESTRICT, l, dev(x), None, yc)
            assert rel(host(yc), c1.P[l].T @ x) < 1e-14
            xc = rng.standard_normal(nc)
            sd.stokes_level_op(h64, sd.STOKES_OP_PROLONG, l, dev(xc), None, y)
            assert rel(host(y), c1.P[l] @ xc) < 1e-14
            # Vanka: weighted sum of patch solves, and one damped sweep
            sd.stokes_level_op(h64, sd.STOKES_OP_VANKA, l, dev(x), None, y)
            assert rel(host(y), o.vanka[l].apply(x)) < 1e-12
            sd.stokes_level_op(h64, sd.STOKES_OP_RELAX, l, dev(x), dev(b), y)
            assert rel(host(y), o.vanka[l].sweep(c1.K[l], x, b, PRM["omega"])) < 1e-12
        else:
            sd.stokes_level_op(h64, sd.STOKES_OP_COARSE, l, dev(b), None, y)
            assert rel(host(y), o.coarse_solve(b)) < 1e-11


def test_vcycle_fp64_matches_oracle(sd, c1, h64):
    o = make_oracle(c1, PRM)
    rng = np.random.default_rng(11)
    for r in (c1.b, rng.standard_normal(c1.b.size)):
        z = torch.empty(r.size, dtype=torch.float64, device="cuda")
        sd.stokes_vcycle(h64, dev(r), z)
        assert rel(host(z), o.apply(r)) < 1e-12


def test_vcycle_fp64_five_levels_matches_oracle(sd):
    """A 64^2 cavity has five levels, so level 3 restricts its residual as
    R b - (R K) x in one launch (R K assembled at setup) and the cycle's
    other fused steps all run; the FP64 cycle equals the oracle's, and so
    does the FP32 cycle to FP32 accuracy."""
    pr = stokes.build_th(M.unit_square(64), bc="lid")
    assert pr.nlevels >= 5
    o = make_oracle(pr, PRM)
    r = np.random.default_rng(41).standard_normal(pr.b.size)
    ref = o.apply(r)
    for prec, tol in ((sd.STOKES_FP64, 1e-12), (sd.STOKES_FP32, 1e-5)):
        h = sd.stokes_setup(pr, dict(PRM, precision=prec))
        sd.stokes_factor_patches(h)
        z = torch.empty(r.size, dtype=torch.float64, device="cuda")
        sd.stokes_vcycle(h, dev(r), z)
        assert rel(host(z), ref) < tol, prec
        sd.stokes_destroy(h)


def test_vcycle_replay_is_bitwise_deterministic(sd, c1, h32):
    r = dev(np.random.default_rng(12).standard_normal(c1.b.size))
    z1 = torch.empty_like(r)
    z2 = torch.empty_like(r)
    sd.stokes_vcycle(h32, r, z1)
    sd.stokes_vcycle(h32, r, z2)
    assert torch.equal(z1, z2)


def test_vcycle_fp32_close_to_oracle(sd, c1, h32):
    o = make_oracle(c1, PRM)
    r = np.random.default_rng(13).standard_normal(c1.b.size)
    z = torch.empty(r.size, dtype=torch.float64, device="cuda")
    sd.stokes_vcycle(h32, dev(r), z)
    assert rel(host(z), o.apply(r)) < 1e-5


@pytest.mark.parametrize("variant", [dict(schedule=1), dict(schedule=2), dict(nu1=2, nu2=2), dict(nu1=0, nu2=1),
                                     dict(eta_u=0.9, eta_p=0.5)])
def test_schedules_and_sweeps_fp64(sd, c1, variant):
    prm = dict(PRM, **variant)
    h = sd.stokes_setup(c1, dict(prm, precision=sd.STOKES_FP64))
    sd.stokes_factor_patches(h)
    o = make_oracle(c1, prm)
    r = np.random.default_rng(14).standard_normal(c1.b.size)
    z = torch.empty(r.size, dtype=torch.float64, device="cuda")
    sd.stokes_vcycle(h, dev(r), z)
    assert rel(host(z), o.apply(r)) < 1e-12


def test_fgmres_fp64_matches_oracle_iterations(sd, c1, h64):
    o = make_oracle(c1, PRM)
    xo, its_o, rr_o = krylov.fgmres(c1.K[0], c1.b, o.apply, rtol=1e-8, restart=30, maxit=200)
    x = torch.zeros(c1.b.size, dtype=torch.float64, device="cuda")
    rc, info = sd.stokes_fgmres_solve(h64, dev(c1.b), x, rtol=1e-8, restart=30, maxit=200)
    its, st, rr = info[0]
    assert rc == sd.STOKES_OK and rr <= 1e-8
    assert abs(its - its_o) <= 1
    assert rel(host(x), xo) < 1e-6


def test_fgmres_fp32_within_two_iterations(sd, c1, h32, h64):
    b = dev(c1.b)
    x64 = torch.zeros_like(b)
    _, i64 = sd.stokes_fgmres_solve(h64, b, x64, rtol=1e-8, restart=30, maxit=200)
    x32 = torch.zeros_like(b)
    rc, i32 = sd.stokes_fgmres_solve(h32, b, x32, rtol=1e-8, restart=30, maxit=200)
    assert rc == sd.STOKES_OK and i32[0][2] <= 1e-8
    assert abs(i32[0][0] - i64[0][0]) <= 2


def test_fgmres_host_entry_point(sd, c1, h32):
    x = np.zeros_like(c1.b)
    rc, info = sd.stokes_fgmres_solve_host(h32, c1.b.copy(), x, rtol=1e-8, restart=30, maxit=200)
    assert rc == sd.STOKES_OK
    assert np.linalg.norm(c1.b - c1.K[0] @ x) <= 1e-8 * np.linalg.norm(c1.b)


def test_zero_rhs_and_restart(sd, c1, h32):
    b = torch.zeros(c1.b.size, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    rc, info = sd.stokes_fgmres_solve(h32, b, x, rtol=1e-8, restart=30, maxit=10)
    assert rc == sd.STOKES_OK and info[0][0] == 0 and float(x.abs().max()) == 0.0
    # a short restart still converges (several restart cycles)
    x = torch.zeros_like(b)
    rc, info = sd.stokes_fgmres_solve(h32, dev(c1.b), x, rtol=1e-8, restart=5, maxit=300)
    assert rc == sd.STOKES_OK and info[0][2] <= 1e-8


def test_batched_instances_of_different_depth(sd):
    probs = [stokes.build_th(M.unit_square(n), nu=nu, bc="noslip", rhs="random_b", seed=77 + n)
             for n, nu in ((6, 0.1), (16, 1.0), (10, 30.0))]
    depths = {p.nlevels for p in probs}
    assert len(depths) > 1
    h = sd.stokes_setup(probs, dict(PRM, precision=sd.STOKES_FP64))
    sd.stokes_factor_patches(h)
    r = np.concatenate([np.random.default_rng(k).standard_normal(p.b.size) for k, p in enumerate(probs)])
    z = torch.empty(r.size, dtype=torch.float64, device="cuda")
    sd.stokes_vcycle(h, dev(r), z)
    zh = host(z)
    o = 0
    for k, p in enumerate(probs):
        n = p.b.size
        assert rel(zh[o:o + n], make_oracle(p, PRM).apply(r[o:o + n])) < 1e-12
        o += n
    # per-instance FGMRES
    b = np.concatenate([p.b for p in probs])
    x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
    h32 = sd.stokes_setup(probs, dict(PRM, precision=sd.STOKES_FP32))
    sd.stokes_factor_patches(h32)
    rc, info = sd.stokes_fgmres_solve(h32, dev(b), x, rtol=1e-8, restart=30, maxit=200)
    assert rc == sd.STOKES_OK
    xh = host(x)
    o = 0
    for k, p in enumerate(probs):
        n = p.b.size
        assert np.linalg.norm(p.b - p.K[0] @ xh[o:o + n]) <= 1e-8 * np.linalg.norm(p.b)
        assert info[k][2] <= 1e-8
        o += n


def test_invalid_patch_is_rejected_on_the_host(sd):
    pr = stokes.build_th(M.unit_square(4), bc="lid")
    pr.patches[0].dof[3] = pr.K[0].shape[0] + 5   # out of range
    with pytest.raises(sd.StokesError) as ei:
        sd.stokes_setup(pr, dict(PRM, precision=sd.STOKES_FP32))
    assert ei.value.code == sd.STOKES_ERR_INVALID_ARG


def test_cycle_before_factorisation_is_an_error(sd, c1):
    h = sd.stokes_setup(c1, dict(PRM, precision=sd.STOKES_FP32))
    r = dev(c1.b)
    with pytest.raises(sd.StokesError) as ei:
        sd.stokes_vcycle(h, r, torch.empty_like(r))
    assert ei.value.code == sd.STOKES_ERR_STATE


@pytest.fixture(scope="module")
def c2():
    return configs.c2()


def test_c2_full_size_fp64_cycle_matches_oracle(sd, c2):
    h = sd.stokes_setup(c2, dict(PRM, precision=sd.STOKES_FP64))
    sd.stokes_factor_patches(h)
    o = make_oracle(c2, PRM)
    r = np.random.default_rng(15).standard_normal(c2.b.size)
    z = torch.empty(r.size, dtype=torch.float64, device="cuda")
    sd.stokes_vcycle(h, dev(r), z)
    assert rel(host(z), o.apply(r)) < 1e-12


def test_c2_full_size_fp32_solve(sd, c2):
    b = dev(c2.b)
    res = {}
    for prec in (sd.STOKES_FP64, sd.STOKES_FP32):
        h = sd.stokes_setup(c2, dict(PRM, precision=prec))
        sd.stokes_factor_patches(h)
        x = torch.zeros_like(b)
        rc, info = sd.stokes_fgmres_solve(h, b, x, rtol=1e-8, restart=30, maxit=400)
        assert rc == sd.STOKES_OK and info[0][2] <= 1e-8
        res[prec] = (info[0][0], host(x))
    assert abs(res[sd.STOKES_FP32][0] - res[sd.STOKES_FP64][0]) <= 2
    # the two solutions agree to the accuracy the 1e-8 residual allows
    assert rel(res[sd.STOKES_FP32][1], res[sd.STOKES_FP64][1]) < 1e-5


def test_ho_amg_cycle_and_solve(sd):
    """HO-AMG (Alg. 1 applied directly to K0): the cycle runs with a general
    R0 = P0^T; FP64 parity and FP32 FGMRES within +-2 iterations."""
    pr = configs.ho_amg_th2d(16)
    prm = dict(configs.HO_AMG_TH2D)
    h64 = sd.stokes_setup(pr, dict(prm, precision=sd.STOKES_FP64))
    sd.stokes_factor_patches(h64)
    o = make_oracle(pr, prm)
    r = np.random.default_rng(16).standard_normal(pr.b.size)
    z = torch.empty(r.size, dtype=torch.float64, device="cuda")
    sd.stokes_vcycle(h64, dev(r), z)
    assert rel(host(z), o.apply(r)) < 1e-12
    _, its_o, _ = krylov.fgmres(pr.K[0], pr.b, o.apply, rtol=1e-8, restart=30, maxit=200)
    h32 = sd.stokes_setup(pr, dict(prm, precision=sd.STOKES_FP32))
    sd.stokes_factor_patches(h32)
    x = torch.zeros(pr.b.size, dtype=torch.float64, device="cuda")
    rc, info = sd.stokes_fgmres_solve(h32, dev(pr.b), x, rtol=1e-8, restart=30, maxit=200)
    assert rc == sd.STOKES_OK and info[0][2] <= 1e-8 and abs(info[0][0] - its_o) <= 2
