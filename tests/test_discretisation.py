"""Pins of the discretisation (Sec. 2): manufactured-solution convergence
rates of Taylor-Hood P2/P1 (velocity O(h^3), pressure O(h^2) in L2) and of
the auxiliary P1isoP2/P1 operator (velocity O(h^2)), exact element
identities, and the divergence theorem on B."""
import numpy as np
import pytest

from problems import fem, mesh as M, stokes
from oracle import direct
from tests.fe_error import l2_error


def _th_errors(n):
    pr = stokes.build_th(M.unit_square(n), bc="noslip", rhs="manufactured", max_levels=2)
    off = pr.field_off[0]
    x = direct.solve_stokes(pr.K[0], pr.b, off, 2, Mp=pr.Mp)
    V = pr.info["V"]
    mesh = pr.info["mesh"]
    u, p = pr.exact["u"], pr.exact["p"]
    b2 = fem.p2_basis(2)
    n2 = pr.info["n2"]
    eu = 0.0
    for c in range(2):
        eu += l2_error(mesh.x, mesh.cells, V.cell_nodes, b2, x[c * n2:(c + 1) * n2],
                       lambda X, c=c: u(X)[:, c]) ** 2
    ep = l2_error(mesh.x, mesh.cells, mesh.cells, fem.p1_basis(2), x[off[2]:off[3]], p)
    return np.sqrt(eu), ep


def test_taylor_hood_manufactured_rates():
    errs = [_th_errors(n) for n in (16, 32, 64)]
    ru = [errs[k][0] / errs[k + 1][0] for k in range(2)]
    rp = [errs[k][1] / errs[k + 1][1] for k in range(2)]
    # O(h^3) velocity; pressure at least O(h^2) (it approaches 4 from above,
    # superconvergent on coarse meshes)
    assert 7.5 < ru[-1] < 8.5, ru
    assert 3.8 < rp[-1] < 5.0, rp


def _p1iso_errors(n):
    """Solve the P1isoP2/P1 system K1 with the load F = M1 f_I (P1 mass on the
    refined mesh) and measure the velocity L2 error on the refined mesh."""
    mesh = M.unit_square(n)
    V = M.P2Space(mesh)
    bnd = M.p2_boundary_nodes(V)
    K1, A1, _ = stokes.p1iso_K1(V, mesh.cells, None, mesh.nv, bnd, 1.0)
    u, p, f = stokes.manufactured_2d()
    fc, _ = M.uniform_refine_cells(V)
    b1 = fem.p1_basis(2)
    M1 = fem.assemble_mass(V.x, fc, fc, fc, fem.mass_tensor(b1, b1, 2), V.n, V.n)
    fv = f(V.x)
    F = []
    for c in range(2):
        fcomp = M1 @ fv[:, c]
        fcomp[bnd] = 0.0
        F.append(fcomp)
    b = np.concatenate(F + [np.zeros(mesh.nv)])
    off = stokes.field_offsets(V.n, mesh.nv, 2)
    x = direct.solve_stokes(K1, b, off, 2)
    e = 0.0
    for c in range(2):
        e += l2_error(V.x, fc, fc, b1, x[c * V.n:(c + 1) * V.n], lambda X, c=c: u(X)[:, c]) ** 2
    return np.sqrt(e)


def test_p1isop2_velocity_rate():
    e = [_p1iso_errors(n) for n in (8, 16, 32)]
    r = e[1] / e[2]
    assert 3.5 < r < 4.6, (e, r)


def test_element_identities():
    for d in (2, 3):
        b2 = fem.p2_basis(d)
        C = fem.stiffness_tensor(b2, d)
        # a random simplex: stiffness rows sum to zero, mass sums to |T|
        x = np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.2, 0.9, 0.1], [0.1, 0.2, 1.1]])[: d + 1, :d]
        cells = np.arange(d + 1)[None, :]
        vol, g = fem.geometry(x, cells)
        G = np.einsum("ckd,cld->ckl", g, g)
        Ke = vol[:, None, None] * np.einsum("ijkl,ckl->cij", C, G)
        assert np.abs(Ke.sum(axis=2)).max() < 1e-13
        E = fem.mass_tensor(b2, b2, d)
        assert abs(E.sum() - 1.0) < 1e-14
        # P2 reproduces the quadratic x0^2: its stiffness energy equals int |grad|^2
        xv = np.concatenate([x, 0.5 * (x[M.EDGES[d][:, 0]] + x[M.EDGES[d][:, 1]])])
        q = xv[:, 0] ** 2
        energy = q @ Ke[0] @ q
        lam_c = np.full(d + 1, 1.0 / (d + 1))
        # int (2 x0)^2 = 4 int x0^2; x0 is linear so x0^2 is integrated exactly
        xl = x[:, 0]
        int_x2 = vol[0] * (np.sum(xl ** 2) + np.sum(np.triu(np.outer(xl, xl), 1))) * 2.0 / ((d + 1) * (d + 2))
        assert abs(energy - 4.0 * int_x2) < 1e-12


def test_divergence_theorem_on_B():
    """sum_q B[q, j] = - int div phi_j = 0 for every interior velocity node."""
    pr = stokes.build_th(M.unit_square(6), bc="lid", max_levels=2)
    off = pr.field_off[0]
    B = pr.K[0][off[2]:off[3], :off[2]]
    colsum = np.asarray(B.sum(axis=0)).ravel()
    assert np.abs(colsum).max() < 1e-13
    # K0 is symmetric and the pressure constant is its null vector
    K = pr.K[0]
    assert abs(K - K.T).max() < 1e-14
    one = np.zeros(K.shape[0])
    one[off[2]:] = 1.0
    assert np.abs(K @ one).max() < 1e-13


def test_scott_vogelius_is_pointwise_divergence_free():
    """On the Alfeld split, div P2 lies in P1disc, so the discrete solution is
    divergence-free to roundoff (Sec. 2.1); Taylor-Hood is not."""
    from problems import stokes as S
    pr = S.build_sv(8, max_levels=2)
    off = pr.field_off[0]
    x = direct.solve_stokes(pr.K[0], pr.b, off, 2, Mp=pr.Mp)
    dn = S.divergence_norm(pr, x)
    A = pr.K[0][: off[2], : off[2]]
    energy = np.sqrt(x[: off[2]] @ (A @ x[: off[2]]))
    assert dn < 1e-12 * energy, (dn, energy)
    # the same measure is clearly nonzero for Taylor-Hood (div u_h in P1disc,
    # measured with a discontinuous-pressure divergence on its own mesh)
    import scipy.sparse.linalg as spla
    th = stokes.build_th(M.unit_square(8), bc="noslip", rhs="manufactured", max_levels=2)
    xo = direct.solve_stokes(th.K[0], th.b, th.field_off[0], 2, Mp=th.Mp)
    mesh, V = th.info["mesh"], th.info["V"]
    pdg = np.arange(3 * mesh.nc).reshape(-1, 3)
    b1, b2 = fem.p1_basis(2), fem.p2_basis(2)
    Bd = fem.assemble_div(mesh.x, mesh.cells, pdg, V.cell_nodes, fem.div_tensor(b1, b2, 2), pdg.size, V.n)
    Md = fem.assemble_mass(mesh.x, mesh.cells, pdg, pdg, fem.mass_tensor(b1, b1, 2), pdg.size, pdg.size)
    n2 = V.n
    Bu = Bd[0] @ xo[:n2] + Bd[1] @ xo[n2:2 * n2]
    dth = np.sqrt(Bu @ spla.spsolve(Md.tocsc(), Bu))
    assert dth > 1e-6, dth


def test_scott_vogelius_transfers():
    """Pi^T M_dg Pi = Mcg (a continuous P1 function is its own projection),
    the perturbed Alfeld mesh stays valid, and the 3-seed cell patches hold
    the 6 P2 nodes of their cell (15 DoFs inside the domain)."""
    from problems import stokes as S
    pr = S.build_sv(8)
    Pi = pr.info["Pi"]
    assert abs(pr.R0p @ Pi - pr.Mcg).max() < 1e-15
    base = pr.info["base"]
    assert M.cell_measure(base.x, base.cells).min() > 0
    pa = pr.patches[0]
    assert np.all(pa.npres == 3) and np.diff(pa.ptr).max() == 15
    # the projection solve: Chebyshev-Jacobi of degree 32 against a direct solve
    from oracle.cycle import chebyshev_jacobi
    import scipy.sparse.linalg as spla
    rhs = np.random.default_rng(0).standard_normal(pr.Mcg.shape[0])
    x = chebyshev_jacobi(pr.Mcg, rhs, 0.5, 2.0, 32)
    xd = spla.spsolve(pr.Mcg.tocsc(), rhs)
    assert np.linalg.norm(x - xd) < 1e-13 * np.linalg.norm(xd)
    # the Wathen interval holds the spectrum of D^-1 Mcg
    D = pr.Mcg.diagonal()
    ev = np.linalg.eigvals(pr.Mcg.toarray() / D[:, None]).real
    assert ev.min() >= 0.5 - 1e-12 and ev.max() <= 2.0 + 1e-12


def test_3d_meshes_and_operators():
    """Kuhn cube and Bey's red refinement: the cells tile the cube, the eight
    children of a tetrahedron have equal volume; the 3D Taylor-Hood K0 is
    symmetric with the pressure constant as null vector, 1^T B = 0 on
    interior velocity columns, and interior patches hold the 65 P2 nodes of a
    vertex star (196 DoFs)."""
    mesh = M.unit_cube(3)
    vol = M.cell_measure(mesh.x, mesh.cells)
    assert abs(vol.sum() - 1.0) < 1e-13 and vol.min() > 0
    V = M.P2Space(mesh)
    fc, _ = M.uniform_refine_cells(V)
    fv = M.cell_measure(V.x, fc).reshape(-1, 8)
    assert np.allclose(fv, vol[:, None] / 8.0, rtol=1e-12)
    pr = stokes.build_th(M.unit_cube(4), bc="lid", max_levels=3)
    K = pr.K[0]
    off = pr.field_off[0]
    assert abs(K - K.T).max() < 1e-14
    one = np.zeros(K.shape[0])
    one[off[3]:] = 1.0
    assert np.abs(K @ one).max() < 1e-13
    B = K[off[3]:off[4], : off[3]]
    assert np.abs(np.asarray(B.sum(axis=0)).ravel()).max() < 1e-13
    assert np.diff(pr.patches[0].ptr).max() == 196
