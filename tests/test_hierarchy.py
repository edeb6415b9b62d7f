"""Pins of the Alg. 1 hierarchy: near-null reproduction by the tentative and
smoothed prolongators, Galerkin symmetry, the coarse pressure null vector,
block-diagonal structure and aggregation coverage."""
import numpy as np
import scipy.sparse as sp

from problems import mesh as M, sa, stokes


def _prob():
    return stokes.build_th(M.unit_square(16), bc="lid")


def test_aggregation_covers_free_nodes_once():
    pr = _prob()
    off = pr.field_off[1]
    A1 = pr.K[1][: off[1], : off[1]]
    excl = sa.isolated_rows(A1)
    agg, na = sa.aggregate(sa.strength(A1), excl)
    assert np.all(agg[excl] == -1)
    assert np.all(agg[~excl] >= 0)
    assert set(np.unique(agg[~excl])) == set(range(na))
    # Dirichlet rows are exactly the boundary nodes
    assert np.array_equal(excl, pr.dirichlet[: off[1]])


def test_near_null_reproduced_by_pressure_interpolation():
    pr = _prob()
    d = pr.dim
    offL = pr.field_off[-1]
    v = pr.coarse_null[offL[d]:offL[d + 1]]
    for l in range(pr.nlevels - 2, 0, -1):
        P = pr.P[l]
        offf, offc = pr.field_off[l], pr.field_off[l + 1]
        # block-diagonal: no velocity-pressure coupling in P
        assert P[offf[d]:, : offc[d]].nnz == 0 and P[: offf[d], offc[d]:].nnz == 0
        v = P[offf[d]:offf[d + 1], offc[d]:offc[d + 1]] @ v
    # the coarse null vector interpolates to the fine pressure constant
    assert np.abs(v - 1.0).max() < 1e-12


def test_galerkin_symmetry_and_coarse_null():
    pr = _prob()
    for l in range(2, pr.nlevels):
        K = pr.K[l]
        assert abs(K - K.T).max() < 1e-12 * abs(K).max()
        Kc = (pr.P[l - 1].T @ pr.K[l - 1] @ pr.P[l - 1]).tocsr()
        assert abs(Kc - K).max() < 1e-12 * abs(K).max()
    KL = pr.K[-1]
    assert np.abs(KL @ pr.coarse_null).max() < 1e-13 * np.abs(KL).max() * np.linalg.norm(pr.coarse_null)


def test_smoothed_prolongator_of_laplacian_keeps_constants():
    """SA on a pure Neumann Laplacian: P B_c = B exactly (A B = 0)."""
    pr = _prob()
    Ap = stokes.pressure_laplacian(pr.info["mesh"])
    Ps, As, Bs = sa.sa_field(Ap, np.ones(Ap.shape[0]), 4)
    for k, P in enumerate(Ps):
        assert np.abs(P @ Bs[k + 1] - Bs[k]).max() < 1e-12


def test_lanczos_matches_dense_eigenvalue():
    A = sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], shape=(40, 40)).tocsr()
    exact = 2.0 - 2.0 * np.cos(40 * np.pi / 41)
    assert abs(sa.lanczos_max(A, steps=40) - exact) < 1e-10


def test_patches_th_structure():
    """Interior TH patches: one pressure seed and the 19 P2 nodes of its
    vertex star per velocity component (39 DoFs); same node list for every
    component; no Dirichlet DoF in any patch."""
    pr = _prob()
    for l in (0, 1):
        pa = pr.patches[l]
        sizes = np.diff(pa.ptr)
        assert sizes.max() == 39
        assert np.all(pa.npres == 1)
        off = pr.field_off[l]
        for i in range(pa.npatch):
            dofs = pa.dof[pa.ptr[i]:pa.ptr[i + 1]]
            m = pa.nvel[i, 0]
            assert np.array_equal(dofs[:m] - off[0], dofs[m:2 * m] - off[1])
            assert not pr.dirichlet[dofs].any()
            assert np.all(np.diff(dofs[:m]) > 0)


def test_ho_amg_hierarchy():
    """Alg. 1 on K0 directly: block-diagonal SA interpolation of the P2
    velocity and P1 pressure, Galerkin coarse operators, null vector."""
    pr = stokes.build_ho_amg(M.unit_square(16), bc="lid")
    assert pr.nlevels >= 3
    for l in range(1, pr.nlevels):
        Kc = (pr.P[l - 1].T @ pr.K[l - 1] @ pr.P[l - 1]).tocsr()
        assert abs(Kc - pr.K[l]).max() < 1e-12 * abs(pr.K[l]).max()
    KL = pr.K[-1]
    assert np.abs(KL @ pr.coarse_null).max() < 1e-12 * np.abs(KL).max() * np.linalg.norm(pr.coarse_null)
