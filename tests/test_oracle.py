"""Pins of the FP64 oracle against facts fixed by the paper and by linear
algebra: the partition of unity of Eq. vanka, the block factorisation of
Eqs. vanka_fact1/2 against dense LU on every patch, a single all-covering
patch against a direct solve, the sampled Vanka application against the full
one, the bordered coarsest solve against its projection property, the
Scott-Vogelius restriction R0 against its projection identity and a direct
mass solve, the two-level form of Eq. TG-operator-full as a dense operator
product for Taylor-Hood and for Scott-Vogelius, the
Chebyshev closed form, FGMRES special cases and its minimisation over the
preconditioned vectors, Krylov-wrapped relaxation, DLSC, and convergence of
the stationary DC iteration."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import cycle, direct, krylov, vanka
from problems import configs, mesh as M, stokes


@pytest.fixture(scope="module")
def c1():
    return configs.c1()


def test_partition_of_unity(c1):
    for l, pa in enumerate(c1.patches):
        n = c1.K[l].shape[0]
        W = vanka.partition_of_unity(pa, n)
        s = np.zeros(n)
        for ix in vanka.patch_lists(pa):
            s[ix] += 1.0
        covered = s > 0
        assert np.allclose((W * s)[covered], 1.0, atol=1e-15)
        # every non-Dirichlet DoF of the assembled levels lies in some patch
        if l <= 1:
            assert np.array_equal(covered, ~c1.dirichlet)


def _block_solve(Kp, m_u, m_p, rhs):
    """x = [I U^; 0 I][A^-1 0; B^ S^-1] b with U = A^-1 B^T, S = -B A^-1 B^T,
    B^ = -S^-1 B A^-1, U^ = -U (Eqs. vanka_fact1/2)."""
    A = Kp[:m_u, :m_u]
    B = Kp[m_u:, :m_u]
    Ainv = np.linalg.inv(A)
    U = Ainv @ B.T
    S = -B @ U
    Sinv = np.linalg.inv(S)
    Bh = -Sinv @ B @ Ainv
    Uh = -U
    y_u = Ainv @ rhs[:m_u]
    y_p = Bh @ rhs[:m_u] + Sinv @ rhs[m_u:]
    return np.concatenate([y_u + Uh @ y_p, y_p])


def test_block_factorisation_equals_dense_lu(c1):
    rng = np.random.default_rng(0)
    worst = 0.0
    for l, pa in enumerate(c1.patches):
        K = c1.K[l].tocsr()
        for i, ix in enumerate(vanka.patch_lists(pa)):
            Kp = K[ix][:, ix].toarray()
            m_p = int(pa.npres[i])
            m_u = ix.size - m_p
            rhs = rng.standard_normal(ix.size)
            x_lu = np.linalg.solve(Kp, rhs)
            x_bf = _block_solve(Kp, m_u, m_p, rhs)
            worst = max(worst, np.linalg.norm(x_bf - x_lu) / np.linalg.norm(x_lu))
            # the velocity block is block diagonal by component (vector Laplacian)
            m = pa.nvel[i, 0]
            assert np.abs(Kp[:m, m:2 * m]).max() == 0.0
    assert worst < 1e-12


def test_sampled_vanka_equals_the_full_application(c1):
    """The sampled Vanka application used for full-size checks (only the
    patches holding the sampled DoFs) gives the full Eq. vanka application
    at those DoFs, on every level."""
    o = cycle.Oracle(c1, cycle.Params(omega=[1.0] * (c1.nlevels - 1)))
    rng = np.random.default_rng(17)
    for l in range(c1.nlevels - 1):
        n = c1.K[l].shape[0]
        r = rng.standard_normal(n)
        full = o.vanka[l].apply(r)
        dofs = np.sort(rng.choice(n, size=min(40, n), replace=False))
        ref = vanka.sampled_apply(c1.K[l], c1.patches[l], r, dofs)
        assert np.abs(ref - full[dofs]).max() <= 1e-12 * np.abs(full).max()


def test_bordered_coarsest_solve(c1):
    """The coarsest solve of the bordered system [K_L n; n^T 0] (n the coarse
    pressure null vector, K_L n = 0): x solves K_L x = b - (n.b / n.n) n, the
    projection of b on the range, and is orthogonal to n."""
    o = cycle.Oracle(c1, cycle.Params(omega=[1.0] * (c1.nlevels - 1)))
    KL = c1.K[-1].toarray()
    n = c1.coarse_null
    assert np.abs(KL @ n).max() <= 1e-10 * np.abs(KL).max() * np.abs(n).max()
    b = np.random.default_rng(23).standard_normal(KL.shape[0])
    x = o.coarse_solve(b)
    proj = b - (n @ b) / (n @ n) * n
    assert np.linalg.norm(KL @ x - proj) <= 1e-10 * np.linalg.norm(b)
    assert abs(n @ x) <= 1e-10 * np.linalg.norm(x) * np.linalg.norm(n)


def test_single_patch_is_a_direct_solve(c1):
    """One patch holding every free DoF except one pressure DoF (which fixes
    the pressure constant): Vanka with W = 1 is an exact solve."""
    K = c1.K[0].tocsr()
    n = K.shape[0]
    off = c1.field_off[0]
    free = np.nonzero(~c1.dirichlet)[0]
    free = free[free != off[2]]
    nv = np.sum(free < off[1])
    pa = stokes.Patches(np.array([0, free.size]), free.astype(np.int32),
                        np.array([[nv, nv]], dtype=np.int32), np.array([off[3] - off[2] - 1], dtype=np.int32))
    vl = vanka.VankaLevel(K, pa)
    rng = np.random.default_rng(1)
    xs = rng.standard_normal(n)
    xs[c1.dirichlet] = 0.0
    r = K @ xs
    z = vl.apply(r)
    ref = xs.copy()
    ref[off[2]:] -= xs[off[2]]
    ref[c1.dirichlet] = 0.0
    assert np.linalg.norm(z - ref) < 1e-10 * np.linalg.norm(ref)


def _dense_vanka(K, pa):
    n = K.shape[0]
    Kd = K.toarray()
    W = vanka.partition_of_unity(pa, n)
    Minv = np.zeros((n, n))
    for ix in vanka.patch_lists(pa):
        Minv[np.ix_(ix, ix)] += np.linalg.inv(Kd[np.ix_(ix, ix)])
    return W[:, None] * Minv


def test_two_level_cycle_is_eq_tg_operator_full():
    """With K1 as the coarsest level (gamma = infinity), one DC application
    has error propagation
    G = (I - w M0^-1 K0)(I - P0 K1^-1 eta R0 K0)(I - w M0^-1 K0)."""
    pr = stokes.build_th(M.unit_square(6), bc="lid", max_levels=2)
    assert pr.nlevels == 2
    par = cycle.Params(eta_u=0.8, eta_p=0.6, omega=[0.55])
    o = cycle.Oracle(pr, par)
    K0 = pr.K[0].toarray()
    K1 = pr.K[1].toarray()
    n = K0.shape[0]
    Minv = _dense_vanka(pr.K[0], pr.patches[0])
    S = np.eye(n) - 0.55 * Minv @ K0
    nvec = pr.coarse_null
    Bd = np.block([[K1, nvec[:, None]], [nvec[None, :], np.zeros((1, 1))]])
    K1inv = np.linalg.inv(Bd)[:n, :n]
    off = pr.field_off[0]
    eta = np.diag(np.concatenate([np.full(off[2], 0.8), np.full(off[3] - off[2], 0.6)]))
    P0 = pr.P[0].toarray()
    G = S @ (np.eye(n) - P0 @ K1inv @ eta @ P0.T @ K0) @ S
    rng = np.random.default_rng(2)
    e = rng.standard_normal(n)
    e[pr.dirichlet] = 0.0
    z = o.apply(K0 @ e)
    free = ~pr.dirichlet
    lhs = (e - z)[free]
    rhs = (G @ e)[free]
    assert np.linalg.norm(lhs - rhs) < 1e-11 * np.linalg.norm(e)


def test_sv_restrict0_returns_a_continuous_pressure_and_the_velocity():
    """Scott-Vogelius R0 (Eq. interp and the pressure transfers of Sec. 3.1):
    velocity injection, and R0^p = Mcg^-1 Pi^T M_dg on the pressure.  Since
    Pi^T M_dg Pi = Mcg, R0 maps (d_u, Pi g) to (d_u, g) for every continuous
    g, up to the degree-32 Chebyshev error of the mass solve; on a general
    discontinuous d_p it is the L2 projection Mcg^-1 (Pi^T M_dg d_p), checked
    against a sparse direct solve."""
    import scipy.sparse.linalg as spla
    pr = stokes.build_sv(4)
    o = cycle.Oracle(pr, cycle.Params(eta_u=1.0, eta_p=2.68, omega=[0.78] + [0.55] * (pr.nlevels - 2)))
    off0, off1 = pr.field_off[0], pr.field_off[1]
    d = pr.dim
    Pi = pr.info["Pi"]
    rng = np.random.default_rng(31)
    du = rng.standard_normal(off0[d])
    g = rng.standard_normal(Pi.shape[1])
    out = o.restrict0(np.concatenate([du, Pi @ g]))
    assert out.size == pr.K[1].shape[0]
    assert off1[d] == off0[d] and np.array_equal(out[: off1[d]], du)
    assert np.linalg.norm(out[off1[d]:] - g) <= 1e-13 * np.linalg.norm(g)
    dp = rng.standard_normal(off0[d + 1] - off0[d])
    out = o.restrict0(np.concatenate([du, dp]))
    ref = spla.spsolve(pr.Mcg.tocsc(), pr.info["Pi"].T @ (pr.info["Mdg"] @ dp))
    assert np.linalg.norm(out[off1[d]:] - ref) <= 1e-13 * np.linalg.norm(ref)


def test_sv_two_level_cycle_is_eq_tg_operator_full():
    """The Scott-Vogelius twin of the two-level identity: with K1 coarsest,
    G = S (I - P0 K1^-1 eta R0 K0) S, S = I - w0 M0^-1 K0 with the 3-seed
    cell patches, P0 = blockdiag(I, Pi), R0 = blockdiag(I, Mcg^-1 Pi^T M_dg)
    formed densely from the definitions (exact mass inverse)."""
    pr = stokes.build_sv(4, max_levels=2)
    assert pr.nlevels == 2
    w0, eu, ep = 0.78, 1.0, 2.68
    o = cycle.Oracle(pr, cycle.Params(eta_u=eu, eta_p=ep, omega=[w0]))
    K0 = pr.K[0].toarray()
    K1 = pr.K[1].toarray()
    n0, n1 = K0.shape[0], K1.shape[0]
    d = pr.dim
    off0 = pr.field_off[0]
    nv = off0[d]
    S = np.eye(n0) - w0 * _dense_vanka(pr.K[0], pr.patches[0]) @ K0
    nvec = pr.coarse_null
    Bd = np.block([[K1, nvec[:, None]], [nvec[None, :], np.zeros((1, 1))]])
    K1inv = np.linalg.inv(Bd)[:n1, :n1]
    Pi = pr.info["Pi"].toarray()
    R0 = np.zeros((n1, n0))
    R0[:nv, :nv] = np.eye(nv)
    R0[nv:, nv:] = np.linalg.solve(pr.Mcg.toarray(), Pi.T @ pr.info["Mdg"].toarray())
    P0 = pr.P[0].toarray()
    assert np.array_equal(P0[nv:, nv:], Pi)
    eta = np.diag(np.concatenate([np.full(nv, eu), np.full(n0 - nv, ep)]))
    G = S @ (np.eye(n0) - P0 @ K1inv @ R0 @ eta @ K0) @ S
    rng = np.random.default_rng(32)
    e = rng.standard_normal(n0)
    e[pr.dirichlet] = 0.0
    z = o.apply(K0 @ e)
    free = ~pr.dirichlet
    assert np.linalg.norm((e - z)[free] - (G @ e)[free]) < 1e-11 * np.linalg.norm(e)


def test_dropping_eta_is_detected():
    """A planted mistake (eta ignored) breaks the two-level identity above."""
    pr = stokes.build_th(M.unit_square(4), bc="lid", max_levels=2)
    par = cycle.Params(eta_u=0.8, eta_p=0.6, omega=[0.55])
    good = cycle.Oracle(pr, par)
    bad = cycle.Oracle(pr, par)
    bad.eta = np.ones_like(bad.eta)
    r = np.random.default_rng(3).standard_normal(pr.K[0].shape[0])
    assert np.linalg.norm(good.apply(r) - bad.apply(r)) > 1e-3 * np.linalg.norm(good.apply(r))


def test_chebyshev_jacobi_closed_form():
    """On an eigenvector of D^-1 M with eigenvalue mu in [a, b] the error of
    the degree-k semi-iteration is T_k((b+a-2mu)/(b-a)) / T_k((b+a)/(b-a))."""
    n = 50
    M_ = sp.diags([-0.5, 2.0, -0.5], [-1, 0, 1], shape=(n, n)).tocsr()  # D^-1 M = I - T/4
    a, b = 0.5, 1.5
    for j in (1, 7, 30):
        mu = 1.0 - 0.5 * np.cos(j * np.pi / (n + 1))
        v = np.sin(j * np.pi * np.arange(1, n + 1) / (n + 1))
        for k in (1, 4, 9):
            x = cycle.chebyshev_jacobi(M_, M_ @ v, a, b, k)
            err = np.linalg.norm(x - v) / np.linalg.norm(v)
            Tk = lambda t: np.cosh(k * np.arccosh(t)) if abs(t) >= 1 else np.cos(k * np.arccos(t))
            pred = abs(Tk((b + a - 2 * mu) / (b - a)) / Tk((b + a) / (b - a)))
            assert abs(err - pred) < 1e-12


def test_fgmres_identity_is_gmres_and_exact_in_n_steps():
    rng = np.random.default_rng(4)
    n = 30
    A = rng.standard_normal((n, n)) + 8 * np.eye(n)
    b = rng.standard_normal(n)
    x, its, rr = krylov.gmres_identity(A, b, rtol=1e-13)
    assert its <= n and rr < 1e-13
    assert np.linalg.norm(x - np.linalg.solve(A, b)) < 1e-11 * np.linalg.norm(x)
    # an exact preconditioner converges in one iteration
    x1, its1, rr1 = krylov.fgmres(A, b, lambda v: np.linalg.solve(A, v), rtol=1e-12)
    assert its1 == 1 and rr1 < 1e-12
    # the residual history of GMRES is monotone
    h = []
    krylov.fgmres(A, b, lambda v: v.copy(), rtol=1e-12, restart=n, history=h)
    assert all(h[k + 1] <= h[k] * (1 + 1e-12) for k in range(len(h) - 1))


def test_stationary_dc_iteration_contracts(c1):
    par = cycle.Params(**{k: v for k, v in configs.TH2D_VANKA.items() if k != "omega"},
                       omega=[configs.TH2D_VANKA["omega"]] * (c1.nlevels - 1))
    o = cycle.Oracle(c1, par)
    K, b = c1.K[0], c1.b
    x = np.zeros_like(b)
    res = []
    for _ in range(25):
        x = x + o.apply(b - K @ x)
        res.append(np.linalg.norm(b - K @ x))
    factor = (res[-1] / res[-11]) ** 0.1
    assert factor < 0.9, factor


def test_fgmres_minimises_over_the_preconditioned_vectors():
    """Flexible GMRES (Sec. 4): with a preconditioner that changes at every
    step, the m-step iterate is x0 + Z y with Z the preconditioner's outputs,
    and its residual is the least-squares minimum of ||b - K (x0 + Z y)||
    over all y (computed here independently of the Arnoldi recurrences)."""
    rng = np.random.default_rng(41)
    n, m = 40, 7
    A = rng.standard_normal((n, n)) + 6 * np.eye(n)
    b = rng.standard_normal(n)
    x0 = rng.standard_normal(n)
    Z = []

    def precond(v):
        # a different, fixed-seed linear map per call: z = (I + 0.3 R_k) v
        R = np.random.default_rng(100 + len(Z)).standard_normal((n, n)) / np.sqrt(n)
        z = v + 0.3 * (R @ v)
        Z.append(z)
        return z

    x, its, rr = krylov.fgmres(A, b, precond, x0=x0, rtol=1e-30, restart=m + 5, maxit=m)
    assert its == m and len(Z) == m
    Zm = np.array(Z).T
    y, *_ = np.linalg.lstsq(A @ Zm, b - A @ x0, rcond=None)
    best = np.linalg.norm(b - A @ (x0 + Zm @ y))
    assert abs(np.linalg.norm(b - A @ x) - best) <= 1e-10 * np.linalg.norm(b)
    # the correction lies in span(Z)
    c, *_ = np.linalg.lstsq(Zm, x - x0, rcond=None)
    assert np.linalg.norm(Zm @ c - (x - x0)) <= 1e-10 * np.linalg.norm(x - x0)
    # a flipped sign in the update (x0 - Z y) would not minimise
    assert np.linalg.norm(b - A @ (x0 - Zm @ y)) > 1.5 * best


def test_fgmres_dc_solves_c1_to_tolerance(c1):
    par = cycle.Params(**{k: v for k, v in configs.TH2D_VANKA.items() if k != "omega"},
                       omega=[configs.TH2D_VANKA["omega"]] * (c1.nlevels - 1))
    o = cycle.Oracle(c1, par)
    x, its, rr = krylov.fgmres(c1.K[0], c1.b, o.apply, rtol=1e-8, restart=30, maxit=100)
    assert rr <= 1e-8 and its <= 20
    xd = direct.solve_stokes(c1.K[0], c1.b, c1.field_off[0], 2, Mp=c1.Mp)
    xz = direct.zero_mean_pressure(x, c1.field_off[0], 2, c1.Mp)
    assert np.linalg.norm(xz - xd) < 1e-6 * np.linalg.norm(xd)


def test_fgmres_dlsc_amg_solves_c1_to_tolerance(c1):
    """DLSC on every level (Mu = diagonal mass on K0): FGMRES reaches the
    direct solution of C1."""
    from tests.helpers import make_oracle
    o = make_oracle(c1, configs.th2d_dlsc(c1.nlevels))
    x, its, rr = krylov.fgmres(c1.K[0], c1.b, o.apply, rtol=1e-8, restart=30, maxit=100)
    assert rr <= 1e-8 and its <= 20
    xd = direct.solve_stokes(c1.K[0], c1.b, c1.field_off[0], 2, Mp=c1.Mp)
    xz = direct.zero_mean_pressure(x, c1.field_off[0], 2, c1.Mp)
    assert np.linalg.norm(xz - xd) < 1e-6 * np.linalg.norm(xd)


def _exact_dlsc(dl, x, rhs, Ai, Sp):
    """One DLSC sweep of dl with exact inner solves (A^-1, and S^+ for the
    Schur operator), by substituting the oracle's Chebyshev routine."""
    from oracle import dlsc

    def solve(op, b, lo, hi, degree, dinv=None):
        return Ai @ b if b.size == Ai.shape[0] else Sp @ b

    orig = dlsc.chebyshev
    dlsc.chebyshev = solve
    try:
        return dl.one(x, rhs)
    finally:
        dlsc.chebyshev = orig


@pytest.mark.parametrize("l", [1, 0])
def test_dlsc_sweep_is_the_factorised_update(l):
    """With exact inner solves, one DLSC sweep (Alg. 2) from x adds
    [I Mu^-1 B^T; 0 -Ap^][A 0; B S]^-1 r, S = B Mu^-1 B^T,
    Ap^ = S^+ (B Mu^-1 A Mu^-1 B^T), the approximate factorisation of
    Sec. 3.3.2 with the derivation's sign; Mu = I on the P1isoP2 level 1 and
    the diagonal of the P2 velocity mass matrix on level 0."""
    from oracle import dlsc
    pr = stokes.build_th(M.unit_square(4), bc="lid", max_levels=3)
    par = cycle.Params(cheb_deg=(3, 3, 6), dlsc_sweeps=1)
    dl = dlsc.DLSCLevel(pr, l, par)
    mi = dl.mu_inv
    assert (l == 0) == (np.ptp(mi) > 0)
    A, B, BT = dl.A.toarray(), dl.B.toarray(), dl.BT.toarray()
    S = B @ (mi[:, None] * BT)
    Sp = np.linalg.pinv(S)
    Ai = np.linalg.inv(A)
    rng = np.random.default_rng(5)
    n = pr.K[l].shape[0]
    x = rng.standard_normal(n)
    rhs = rng.standard_normal(n)
    xn = _exact_dlsc(dl, x, rhs, Ai, Sp)
    r = rhs - pr.K[l] @ x
    nv = dl.nv
    ru, rp = r[:nv], r[nv:]
    v = Ai @ ru
    q = Sp @ (rp - B @ v)
    Ap = Sp @ (B @ (mi[:, None] * (A @ (mi[:, None] * BT))))
    upd = np.concatenate([v + mi * (BT @ q), -Ap @ q])
    assert np.linalg.norm((xn - x) - upd) < 1e-10 * np.linalg.norm(upd)


def test_dlsc_exact_sweep_meets_continuity_and_the_least_squares_commutator():
    """A property of the method, not of its formula: with exact inner solves
    one DLSC sweep on K0 (Mu = diagonal of the P2 velocity mass matrix) for a
    consistent right-hand side leaves (i) a zero continuity residual (the
    velocity correction makes B u = g) and (ii) a momentum residual r_u with
    B Mu^-1 r_u = 0: Ap^ is the least-squares commutator of Sec. 3.3.2,
    whose error A Mu^-1 B^T - B^T Ap^ is Mu^-1-orthogonal to range(B^T).
    Dropping Mu^-1 anywhere, or the plus sign of Eq. fulldlsc, breaks (ii)."""
    from oracle import dlsc
    pr = stokes.build_th(M.unit_square(4), bc="lid", max_levels=3)
    dl = dlsc.DLSCLevel(pr, 0, cycle.Params(cheb_deg=(3, 3, 6), dlsc_sweeps=1))
    mi = dl.mu_inv
    A, B, BT = dl.A.toarray(), dl.B.toarray(), dl.BT.toarray()
    Sp = np.linalg.pinv(B @ (mi[:, None] * BT))
    Ai = np.linalg.inv(A)
    K = pr.K[0]
    rng = np.random.default_rng(7)
    n = K.shape[0]
    rhs = K @ rng.standard_normal(n)          # consistent: b in range(K)
    x = rng.standard_normal(n)
    xn = _exact_dlsc(dl, x, rhs, Ai, Sp)
    res = rhs - K @ xn
    nv = dl.nv
    scale = np.linalg.norm(rhs - K @ x)
    assert np.linalg.norm(res[nv:]) < 1e-10 * scale
    comm = B @ (mi * res[:nv])
    assert np.linalg.norm(comm) < 1e-10 * np.linalg.norm(B @ (mi * (rhs - K @ x)[:nv]))
    assert np.linalg.norm(res[:nv]) > 1e-6 * scale  # not an exact solve: (ii) is a real condition


def test_dlsc_relaxation_reduces_the_error():
    """Two DLSC sweeps with the Table lsd_dgs_config degrees on K1 of a small
    cavity reduce the error of a smooth-plus-random initial guess."""
    from oracle import dlsc
    pr = stokes.build_th(M.unit_square(8), bc="noslip", max_levels=3)
    l = 1
    par = cycle.Params(cheb_deg=(3, 3, 6), dlsc_sweeps=2)
    dl = dlsc.DLSCLevel(pr, l, par)
    K = pr.K[l]
    rng = np.random.default_rng(6)
    xs = rng.standard_normal(K.shape[0])
    xs[pr.dirichlet] = 0.0
    b = K @ xs
    x = dl.sweep(np.zeros_like(b), b)
    assert np.linalg.norm(b - K @ x) < np.linalg.norm(b)


# -- Krylov-wrapped relaxation (Sec. 3.3.1) ---------------------------------

def _rand_system(n, seed):
    rng = np.random.default_rng(seed)
    K = np.eye(n) * 4.0 + rng.standard_normal((n, n)) * 0.3
    M = np.eye(n) * 0.25 + rng.standard_normal((n, n)) * 0.02
    return K, M, rng


def test_krylov_relax_identity_operator_is_exact_in_one_step():
    rng = np.random.default_rng(7)
    n = 9
    x = rng.standard_normal(n)
    b = rng.standard_normal(n)
    out = cycle.krylov_relax(np.eye(n), x, b, lambda v: v, 1)
    assert np.allclose(out, b, atol=1e-14)


def test_krylov_relax_one_step_is_the_residual_minimising_damping():
    """One FGMRES step is x + w* M r with w* = (r, KMr) / (KMr, KMr)."""
    K, M, rng = _rand_system(12, 1)
    x = rng.standard_normal(12)
    b = rng.standard_normal(12)
    r = b - K @ x
    z = M @ r
    Kz = K @ z
    w = (r @ Kz) / (Kz @ Kz)
    out = cycle.krylov_relax(K, x, b, lambda v: M @ v, 1)
    assert np.allclose(out, x + w * z, rtol=1e-13, atol=1e-13)


def test_krylov_relax_two_steps_minimise_over_the_search_space():
    """The result's residual is no larger than that of any combination of the
    two preconditioned directions z1 = M v1, z2 = M v2."""
    K, M, rng = _rand_system(15, 2)
    x = rng.standard_normal(15)
    b = rng.standard_normal(15)
    out = cycle.krylov_relax(K, x, b, lambda v: M @ v, 2)
    r = b - K @ x
    v1 = r / np.linalg.norm(r)
    z1 = M @ v1
    w = K @ z1
    w = w - (w @ v1) * v1
    v2 = w / np.linalg.norm(w)
    z2 = M @ v2
    best = np.linalg.norm(b - K @ out)
    for _ in range(300):
        a, c = rng.standard_normal(2) * 3.0
        assert best <= np.linalg.norm(b - K @ (x + a * z1 + c * z2)) * (1 + 1e-12)
    # and it attains the least-squares optimum over span{z1, z2}
    Z = np.stack([z1, z2], axis=1)
    y = np.linalg.lstsq(K @ Z, r, rcond=None)[0]
    assert abs(best - np.linalg.norm(r - K @ Z @ y)) <= 1e-12 * np.linalg.norm(r)


def test_krylov_relax_n_steps_unpreconditioned_is_a_direct_solve():
    K, _, rng = _rand_system(8, 3)
    x = rng.standard_normal(8)
    b = rng.standard_normal(8)
    out = cycle.krylov_relax(K, x, b, lambda v: v, 8)
    assert np.allclose(K @ out, b, atol=1e-10)


def test_fgmres_with_krylov_wrapped_relaxation_solves_c1(c1):
    nrel = c1.nlevels - 1
    prm = cycle.Params(nu1=2, nu2=2, eta_u=1.0, eta_p=1.0, relax=[cycle.VANKA_KRYLOV] * nrel)
    orc = cycle.Oracle(c1, prm)
    x, its, rel = krylov.fgmres(c1.K[0], c1.b, orc.apply, rtol=1e-8, restart=30, maxit=100)
    assert rel <= 1e-8 and its <= 30
