"""Device steps of the smoothed-aggregation setup (Alg. 1, Sec. 3.2) and of
the Galerkin-level Vanka patch lists (Sec. 3.3.1) against the host setup
step that builds the hierarchies the solve path consumes: strength pattern,
tentative prolongator of the host's aggregates, Jacobi-smoothed prolongator
(with the host's damping) and patch lists.  Index outputs must be equal;
values equal up to the last bits of a different but fixed summation order."""
import numpy as np
import pytest
import scipy.sparse as sp

from problems import mesh as M
from problems import rng, sa, stokes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sd():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2306_06795_gb300 as sd
    return sd


@pytest.fixture(scope="module")
def th2():
    return stokes.build_th(M.unit_square(64), bc="lid")


@pytest.fixture(scope="module")
def th3():
    return stokes.build_th(M.unit_cube(8), bc="lid")


def velocity_blocks(pr):
    """Component-0 velocity blocks of the K1 hierarchy (the scalar operators
    the SA setup coarsens), levels 1 .. L-1."""
    out = []
    for l in range(1, pr.nlevels):
        off = pr.field_off[l]
        out.append(pr.K[l][off[0]:off[1], off[0]:off[1]].tocsr())
    return out


def same_pattern(A, B):
    A, B = A.tocsr(), B.tocsr()
    A.sort_indices()
    B.sort_indices()
    return A.shape == B.shape and np.array_equal(A.indptr, B.indptr) and np.array_equal(A.indices, B.indices)


@pytest.mark.parametrize("theta", [0.0, 0.25])
def test_strength_pattern_equals_host(sd, th2, th3, theta):
    for A in velocity_blocks(th2) + velocity_blocks(th3):
        S = sd.stokes_sa_strength(A, theta)
        assert same_pattern(S, sa.strength(A, theta))
        assert np.all(S.data == 1.0)


def test_tentative_prolongator_equals_host(sd, th2, th3):
    for k, A in enumerate(velocity_blocks(th2) + velocity_blocks(th3)):
        excl = sa.isolated_rows(A)
        agg, na = sa.aggregate(sa.strength(A), excl)
        B = rng.uniform(700 + k, A.shape[0], 0.5, 1.5)
        T_h, Bc_h = sa.tentative(agg, na, B)
        T_d, Bc_d = sd.stokes_sa_tentative(agg, na, B)
        assert same_pattern(T_d, T_h)
        assert np.array_equal(T_d.data, T_h.tocsr().data)
        assert np.array_equal(Bc_d, Bc_h)
        # T Bc = B on aggregated rows
        assert np.allclose((T_d @ Bc_d)[agg >= 0], B[agg >= 0], rtol=1e-14, atol=0)


def test_smoothed_prolongator_matches_host(sd, th2, th3):
    for A in velocity_blocks(th2) + velocity_blocks(th3):
        excl = sa.isolated_rows(A)
        agg, na = sa.aggregate(sa.strength(A), excl)
        T, _ = sa.tentative(agg, na, np.ones(A.shape[0]))
        omega = (4.0 / 3.0) / sa.rho_DinvA(A, ~excl)
        P_h = sa.smooth_prolongator(A, T, excl)
        P_d = sd.stokes_sa_smooth(A, T, omega)
        assert same_pattern(P_d, P_h)
        scale = np.abs(P_h.data).max()
        assert np.abs(P_d.data - P_h.tocsr().data).max() <= 1e-15 * scale


def test_device_steps_rebuild_the_hierarchy(sd, th2):
    """Strength, tentative and smoothed prolongator on the device plus the
    device Galerkin product reproduce the host's next level (host
    aggregation and damping)."""
    A = velocity_blocks(th2)[0]
    excl = sa.isolated_rows(A)
    S = sd.stokes_sa_strength(A)
    agg, na = sa.aggregate(S, excl)
    T, _ = sd.stokes_sa_tentative(agg, na, np.ones(A.shape[0]))
    P = sd.stokes_sa_smooth(A, T, (4.0 / 3.0) / sa.rho_DinvA(A, ~excl))
    Ac = sd.stokes_galerkin(A, P)
    Ps, As, _ = sa.sa_field(A, np.ones(A.shape[0]), max_levels=2)
    assert same_pattern(P, Ps[0])
    assert same_pattern(Ac, As[1])
    assert np.abs((Ac - As[1]).data).max() <= 1e-13 * np.abs(As[1].data).max()


def test_galerkin_level_patches_equal_host(sd, th2, th3):
    n = 0
    for pr in (th2, th3):
        for l in range(2, pr.nlevels - 1):
            ptr, dof, nvel, npres = sd.stokes_vanka_patches(pr.K[l], pr.field_off[l], pr.dim)
            ref = pr.patches[l]
            assert np.array_equal(ptr, ref.ptr)
            assert np.array_equal(dof, ref.dof)
            assert np.array_equal(nvel, ref.nvel)
            assert np.array_equal(npres, ref.npres)
            n += 1
        # level 1 by the algebraic rule as well
        ref1 = stokes.make_patches(pr.K[1], pr.field_off[1], pr.dim)
        ptr, dof, nvel, npres = sd.stokes_vanka_patches(pr.K[1], pr.field_off[1], pr.dim)
        assert np.array_equal(ptr, ref1.ptr) and np.array_equal(dof, ref1.dof)
    assert n >= 2


def test_setup_arguments_are_checked(sd):
    A = sp.identity(4, format="csr")
    with pytest.raises(RuntimeError):
        sd.stokes_sa_strength(A, -1.0)
    with pytest.raises(RuntimeError):
        sd.stokes_sa_tentative(np.array([0, 0, 2, -1]), 2, np.ones(4))  # aggregate 2 out of range
    with pytest.raises(RuntimeError):
        sd.stokes_sa_tentative(np.array([0, 0, 0, -1]), 2, np.ones(4))  # aggregate 1 empty
    with pytest.raises(RuntimeError):
        sd.stokes_vanka_patches(A, np.array([0, 1, 2, 5]), 2)  # offsets do not span K
