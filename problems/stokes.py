"""Seeded synthetic Stokes problems and their solver hierarchies.

``build_problem(name, ...)`` returns a :class:`Problem` holding everything
the solve phase consumes: the high-order operator K0 (Taylor-Hood P2/P1 or
Scott-Vogelius P2/P1disc, Eq. saddle), the low-order P1isoP2/P1 operator K1
(Sec. 3.1), the Alg. 1 smoothed-aggregation hierarchy K2, K3, ... with its
block-diagonal interpolation operators, the transfer P0 between K0 and K1
(Eq. interp), Vanka patch index lists for every relaxed level (Sec. 3.3.1),
the right-hand side and the pressure null vector of the coarsest level.

This is the host setup step: it holds no solve-phase arithmetic (no
relaxation, patch solve, cycle or Krylov method).
"""
from dataclasses import dataclass, field
import numpy as np
import scipy.sparse as sp

from . import fem, mesh as M, rng, sa

TH, SV = 0, 1


@dataclass
class Patches:
    """Vanka patches of one level.  Patch i owns dof[ptr[i]:ptr[i+1]]:
    x-velocity DoFs ascending, then y (then z), then pressure seeds."""
    ptr: np.ndarray
    dof: np.ndarray
    nvel: np.ndarray   # (npatch, dim) velocity DoFs per component
    npres: np.ndarray  # (npatch,)

    @property
    def npatch(self):
        return self.ptr.size - 1


@dataclass
class Problem:
    name: str
    dim: int
    disc: int                      # TH or SV
    nu: float
    K: list                        # K[l], scipy CSR, FP64
    P: list                        # P[l] maps level l+1 to level l
    field_off: list                # per level: array(dim+2) of DoF offsets
    patches: list                  # per relaxed level 0..L-2
    b: np.ndarray                  # right-hand side on level 0
    coarse_null: np.ndarray        # null vector of K[L-1] (pressure constant)
    dirichlet: np.ndarray          # level-0 Dirichlet mask (velocity rows)
    Mp: sp.csr_matrix = None       # pressure mass matrix on level 0
    R0p: sp.csr_matrix = None      # SV: Pi^T M_dg  (n_cg x n_dg)
    Mcg: sp.csr_matrix = None      # SV: P1 mass matrix of the K1 pressure
    mcg_bounds: tuple = (0.5, 2.0)  # Wathen interval of D^-1 Mcg
    lambda_A: np.ndarray = None    # per level, DLSC Chebyshev bounds
    lambda_S: np.ndarray = None
    Mu_diag: np.ndarray = None     # diagonal of the level-0 velocity mass matrix (DLSC on K0)
    exact: dict = field(default_factory=dict)
    info: dict = field(default_factory=dict)

    @property
    def nlevels(self):
        return len(self.K)

    def n(self, l=0):
        return self.K[l].shape[0]


# --------------------------------------------------------------- helpers
def _csr(m):
    m = sp.csr_matrix(m)
    m.sort_indices()
    return m


def _blockdiag(blocks):
    return _csr(sp.block_diag(blocks, format="csr"))


def saddle(Ablocks, Bblocks):
    """K = [A B^T; B 0] with A = blockdiag(Ablocks), B = [B_x B_y (B_z)]."""
    d = len(Ablocks)
    rows = []
    for c in range(d):
        row = [None] * (d + 1)
        row[c] = Ablocks[c]
        row[d] = Bblocks[c].T
        rows.append(row)
    rows.append(list(Bblocks) + [None])
    K = sp.bmat(rows, format="csr")
    return _csr(K)


def drop_columns(B, mask):
    """Remove the columns in mask from B's pattern (explicit zeros kept)."""
    B = B.tocoo()
    k = ~mask[B.col]
    out = sp.csr_matrix((B.data[k], (B.row[k], B.col[k])), shape=B.shape)
    out.sort_indices()
    return out


def nonzero_only(m):
    m = _csr(m.copy())
    m.eliminate_zeros()
    return m


def dirichlet_eliminate(A, Bs, mask, uD, F=None):
    """Symmetric elimination of Dirichlet nodes: identity rows/columns in
    each velocity block, B's Dirichlet columns removed from its pattern,
    RHS lifted."""
    d = len(Bs)
    keep = sp.diags((~mask).astype(float))
    A_in = _csr(keep @ A @ keep + sp.diags(mask.astype(float)))
    A_in.eliminate_zeros()
    Bs_in = []
    g = np.zeros(Bs[0].shape[0])
    Fout = None if F is None else []
    for c in range(d):
        g -= Bs[c] @ (uD[c] * mask)
        Bs_in.append(drop_columns(Bs[c], mask))
        if F is not None:
            f = F[c] - A @ (uD[c] * mask)
            f[mask] = uD[c][mask]
            Fout.append(f)
    return A_in, Bs_in, Fout, g


# --------------------------------------------------------------- assembly
def taylor_hood_K0(mesh, nu, bc, rhs_fn=None, f_nodal=None):
    """P2/P1 operator on ``mesh`` with Dirichlet velocity on the whole
    boundary.  bc: 'lid' (u = (1, 0[, 0]) strictly inside the top edge/face,
    walls win elsewhere) or 'noslip'."""
    d = mesh.dim
    V = M.P2Space(mesh)
    n2 = V.n
    npres = mesh.nv
    b2 = fem.p2_basis(d)
    b1 = fem.p1_basis(d)
    C2 = fem.stiffness_tensor(b2, d)
    A = fem.assemble_stiffness(V.mesh.x, mesh.cells, V.cell_nodes, C2, n2, coef=nu)
    D = fem.div_tensor(b1, b2, d)
    Bs = fem.assemble_div(mesh.x, mesh.cells, mesh.cells, V.cell_nodes, D, npres, n2)
    bnd = M.p2_boundary_nodes(V)
    uD = boundary_values(V.key, V.scale, bnd, bc, d)
    E = fem.mass_tensor(b2, b2, d)
    Mu = fem.assemble_mass(mesh.x, mesh.cells, V.cell_nodes, V.cell_nodes, E, n2, n2)
    F = [np.zeros(n2) for _ in range(d)]
    if rhs_fn is not None:
        fv = rhs_fn(V.x)
        F = [Mu @ fv[:, c] for c in range(d)]
    if f_nodal is not None:
        F = [Mu @ f_nodal[c] for c in range(d)]
    A_in, B_in, F_in, g = dirichlet_eliminate(A, Bs, bnd, uD, F)
    K0 = saddle([A_in] * d, [nonzero_only(B) for B in B_in])
    b = np.concatenate(F_in + [g])
    Mp = fem.assemble_mass(mesh.x, mesh.cells, mesh.cells, mesh.cells, fem.mass_tensor(b1, b1, d), npres, npres)
    return dict(K=K0, b=b, V=V, bnd=bnd, Mu=Mu, Mp=Mp, n2=n2, npres=npres, uD=uD, Bpat=B_in)


def boundary_values(key, scale, bnd, bc, d):
    uD = [np.zeros(key.shape[0]) for _ in range(d)]
    if bc == "lid":
        top = key[:, d - 1] == scale
        inner = np.ones(key.shape[0], dtype=bool)
        for c in range(d - 1):
            inner &= (key[:, c] > 0) & (key[:, c] < scale)
        uD[0][bnd & top & inner] = 1.0
    elif bc != "noslip":
        raise ValueError(bc)
    return uD


def p1iso_K1(V, pcells, pbary_fn, npres, bnd, nu):
    """P1isoP2/P1 operator (Sec. 2.1, 3.1): P1 velocity on R_U of the
    pressure mesh, on the P2 node numbering of ``V``; pressure P1 on the
    coarse cells ``pcells`` (pressure DoF numbers per coarse cell).  The
    divergence integral is exact: div v is constant on a fine cell and the
    coarse pressure is linear, so it is evaluated at the fine centroid."""
    d = V.mesh.dim
    fcells, bary = M.uniform_refine_cells(V)
    nch = bary.shape[0]
    b1 = fem.p1_basis(d)
    C1 = fem.stiffness_tensor(b1, d)
    A = fem.assemble_stiffness(V.x, fcells, fcells, C1, V.n, coef=nu)
    vol, g = fem.geometry(V.x, fcells)
    # parent barycentrics of each child's centroid: nch x (d+1)
    cb = bary.mean(axis=1)
    cbt = np.tile(cb, (pcells.shape[0], 1))       # per fine cell
    pdofs = np.repeat(pcells, nch, axis=0)         # coarse pressure dofs per fine cell
    Bs = []
    nb = d + 1
    r = np.repeat(pdofs, nb, axis=1)
    c = np.tile(fcells, (1, nb))
    for comp in range(d):
        Be = -vol[:, None, None] * cbt[:, :, None] * g[:, None, :, comp]
        Bs.append(fem._coo(r, c, Be.reshape(len(fcells), -1), (npres, V.n), keep_zeros=True))
    zero = [np.zeros(V.n)] * d
    A_in, B_in, _, _ = dirichlet_eliminate(A, Bs, bnd, zero)
    return saddle([A_in] * d, [nonzero_only(B) for B in B_in]), A_in, B_in


def pressure_laplacian(mesh):
    b1 = fem.p1_basis(mesh.dim)
    C1 = fem.stiffness_tensor(b1, mesh.dim)
    return fem.assemble_stiffness(mesh.x, mesh.cells, mesh.cells, C1, mesh.nv)


# --------------------------------------------------------------- hierarchy
def field_offsets(nvel, npres, d):
    return np.array([c * nvel for c in range(d + 1)] + [d * nvel + npres], dtype=np.int64)


class HostSteps:
    """The steps of Alg. 1 the setup route takes, on the host (the default):
    the scalar SA hierarchy of one field, the Galerkin product and the
    Vanka patch lists of a Galerkin level.  A device route supplies the same
    three methods (see problems/device_setup.py)."""

    @staticmethod
    def sa_field(A, B, max_levels, max_coarse):
        return sa.sa_field(A, B, max_levels, max_coarse)

    @staticmethod
    def galerkin(K, P):
        return _csr(P.T @ K @ P)

    @staticmethod
    def patches(K, off, d):
        return make_patches(K, off, d)


def build_hierarchy(K1, A1, Ap, d, nvel1, npres1, max_levels, max_coarse, steps=HostSteps):
    """Alg. 1: scalar SA per field (each velocity component on its block of
    K1, pressure on the auxiliary Laplacian Ap), l_max = min over fields,
    block-diagonal P_l and Galerkin K_{l+1} = P_l^T K_l P_l.  Returns the K1
    hierarchy (K1, K2, ...), the P_l and the pressure near-null vectors."""
    Pv, Av, Bv = steps.sa_field(A1, np.ones(nvel1), max_levels, max_coarse)
    Pp, Ap_, Bp = steps.sa_field(Ap, np.ones(npres1), max_levels, max_coarse)
    # identical scalar blocks per component give identical hierarchies
    lmax = min(len(Av), len(Ap_))
    Ks, Ps, offs = [K1], [], [field_offsets(nvel1, npres1, d)]
    for l in range(lmax - 1):
        P = _blockdiag([Pv[l]] * d + [Pp[l]])
        Kc = steps.galerkin(Ks[-1], P)
        Ps.append(P)
        Ks.append(Kc)
        offs.append(field_offsets(Pv[l].shape[1], Pp[l].shape[1], d))
    return Ks, Ps, offs, Bp[: lmax]


def make_patches(K, off, d, seeds=None, rel_tol=1e-14, exclude=None, Bpattern=None):
    """Algebraic Vanka patches (Sec. 3.3.1): each patch holds its seed
    pressure DoF(s) and every velocity DoF linked to them by an entry of B.
    On assembled levels ``Bpattern`` (per component, element connectivity
    with Dirichlet columns removed) gives the links; on Galerkin levels an
    entry links when |b_ij| > rel_tol * max_j |b_ij|.  A velocity node enters
    with all its components when any component links, so every component of
    a patch has the same node list.  ``seeds`` lists seed groups (default:
    one group per pressure DoF)."""
    K = K.tocsr()
    p0, p1 = off[d], off[d + 1]
    nvel = off[1] - off[0]
    if Bpattern is not None:
        comps = [abs(B).tocsr() for B in Bpattern]
        # structural: every stored entry links, whatever its value
        comps = [sp.csr_matrix((np.ones_like(B.data), B.indices, B.indptr), shape=B.shape) for B in comps]
    else:
        absB = abs(K[p0:p1, : off[d]].tocsr())
        comps = [absB[:, off[c]: off[c + 1]] for c in range(d)]
    mag = comps[0]
    for c in range(1, d):
        mag = mag.maximum(comps[c])
    mag = mag.tocsr()
    rowmax = np.zeros(p1 - p0)
    nz = np.diff(mag.indptr) > 0
    rowmax[nz] = np.maximum.reduceat(mag.data, mag.indptr[:-1][nz]) if mag.nnz else 0
    if seeds is None:
        seeds = np.arange(p1 - p0).reshape(-1, 1)
    ptr = [0]
    dofs = []
    nv = []
    npr = []
    for grp in seeds:
        nodes = set()
        for s in grp:
            a, b = mag.indptr[s], mag.indptr[s + 1]
            cols = mag.indices[a:b]
            vals = mag.data[a:b]
            thr = rel_tol * rowmax[s]
            nodes.update(cols[vals > thr].tolist())
        nodes = np.array(sorted(nodes), dtype=np.int64)
        if exclude is not None and nodes.size:
            nodes = nodes[~exclude[nodes]]
        for c in range(d):
            dofs.append(off[c] + nodes)
        dofs.append(p0 + np.sort(np.asarray(grp, dtype=np.int64)))
        nv.append([nodes.size] * d)
        npr.append(len(grp))
        ptr.append(ptr[-1] + d * nodes.size + len(grp))
    return Patches(np.array(ptr, dtype=np.int64), np.concatenate(dofs).astype(np.int32),
                   np.array(nv, dtype=np.int32), np.array(npr, dtype=np.int32))


def dlsc_bounds(K, field_off, d, steps=20, seed=4242, mu_diag0=None):
    """Largest-eigenvalue estimates of the velocity block A and of
    B Mu^-1 B^T on every level, by seeded Lanczos (the Chebyshev intervals
    of the DLSC stages, Table lsd_dgs_config).  Mu is diag(mu_diag0) on
    level 0 when given (the P2/P1 grid, Sec. 3.3.2), the identity elsewhere."""
    lamA, lamS = [], []
    for l, Kl in enumerate(K):
        off = field_off[l]
        nv = off[d]
        A = Kl[:nv, :nv].tocsr()
        B = Kl[nv:, :nv].tocsr()
        lamA.append(sa.lanczos_max(A, steps=steps, seed=seed + l))
        if l == 0 and mu_diag0 is not None:
            S = (B @ sp.diags(1.0 / mu_diag0) @ B.T).tocsr()
        else:
            S = (B @ B.T).tocsr()
        lamS.append(sa.lanczos_max(S, steps=steps, seed=seed + 100 + l))
    return np.array(lamA), np.array(lamS)


# --------------------------------------------------------------- problems
def manufactured_2d(nu=1.0):
    """u = curl psi, psi = sin^2(pi x) sin^2(pi y); p = cos(pi x) cos(pi y);
    f = -nu lap u + grad p."""
    pi = np.pi

    def u(x):
        X, Y = x[:, 0], x[:, 1]
        return np.stack([pi * np.sin(pi * X) ** 2 * np.sin(2 * pi * Y),
                         -pi * np.sin(2 * pi * X) * np.sin(pi * Y) ** 2], axis=1)

    def p(x):
        return np.cos(pi * x[:, 0]) * np.cos(pi * x[:, 1])

    def f(x):
        X, Y = x[:, 0], x[:, 1]
        lap1 = 2 * pi ** 3 * np.sin(2 * pi * Y) * (2 * np.cos(2 * pi * X) - 1)
        lap2 = -2 * pi ** 3 * np.sin(2 * pi * X) * (2 * np.cos(2 * pi * Y) - 1)
        return np.stack([-nu * lap1 - pi * np.sin(pi * X) * np.cos(pi * Y),
                         -nu * lap2 - pi * np.cos(pi * X) * np.sin(pi * Y)], axis=1)

    return u, p, f


def build_ho_amg(mesh, nu=1.0, bc="lid", rhs="zero", seed=None, max_levels=10, max_coarse=50, name="ho-amg"):
    """HO-AMG (the remark in Sec. 3.2): Alg. 1 applied directly to the
    Taylor-Hood operator K0 - scalar SA on each velocity block of K0 and on
    the P1 pressure Laplacian, block-diagonal P_l, Galerkin coarse operators.
    The cycle is then the standard V-cycle on K0 (eta = 1, R0 = P0^T)."""
    d = mesh.dim
    exact = {}
    rhs_fn = None
    if rhs == "manufactured":
        u, p, f = manufactured_2d(nu)
        rhs_fn = f
        exact = dict(u=u, p=p)
    k0 = taylor_hood_K0(mesh, nu, bc, rhs_fn=rhs_fn)
    V, n2, npres, bnd = k0["V"], k0["n2"], k0["npres"], k0["bnd"]
    A0 = k0["K"][:n2, :n2].tocsr()
    Ap = pressure_laplacian(mesh)
    Ks, Ps, offs, Bp = build_hierarchy(k0["K"], A0, Ap, d, n2, npres, max_levels, max_coarse)
    K, P, field_off = Ks, Ps, offs
    bpat = {0: k0["Bpat"]}
    patches = [make_patches(K[l], field_off[l], d, Bpattern=bpat.get(l)) for l in range(len(K) - 1)]
    L = len(K)
    cn = np.zeros(K[-1].shape[0])
    offL = field_off[-1]
    cn[offL[d]:offL[d + 1]] = Bp[L - 1]
    prob = Problem(name=name, dim=d, disc=TH, nu=nu, K=K, P=P, field_off=field_off, patches=patches, b=k0["b"],
                   coarse_null=cn, dirichlet=np.concatenate([bnd] * d + [np.zeros(npres, bool)]), Mp=k0["Mp"],
                   exact=exact)
    prob.lambda_A, prob.lambda_S = dlsc_bounds(K, field_off, d)
    prob.info = dict(mesh=mesh, V=V, n2=n2, npres=npres, Mu=k0["Mu"], ho_amg=True)
    return prob


def build_th(mesh, nu=1.0, bc="lid", rhs="zero", seed=None, max_levels=10,
             max_coarse=50, name="th", steps=HostSteps):
    """Taylor-Hood P2/P1 K0 with its P1isoP2/P1 K1 and the Alg. 1 hierarchy
    (built by `steps`: HostSteps, or a device route)."""
    d = mesh.dim
    exact = {}
    rhs_fn = None
    if rhs == "manufactured":
        assert d == 2
        u, p, f = manufactured_2d(nu)
        rhs_fn = f
        exact = dict(u=u, p=p)
    k0 = taylor_hood_K0(mesh, nu, bc, rhs_fn=rhs_fn)
    V, n2, npres, bnd = k0["V"], k0["n2"], k0["npres"], k0["bnd"]
    b = k0["b"]
    if rhs == "random_b":
        # i.i.d. N(0,1) on free velocity rows, zero on Dirichlet rows, b_p = 0
        z = rng.normal(seed, d * n2)
        b = np.zeros(d * n2 + npres)
        for c in range(d):
            zc = z[c * n2:(c + 1) * n2].copy()
            zc[bnd] = 0.0
            b[c * n2:(c + 1) * n2] = zc
    K1, A1, B1pat = p1iso_K1(V, mesh.cells, None, npres, bnd, nu)
    Ap = pressure_laplacian(mesh)
    Ks, Ps, offs, Bp = build_hierarchy(K1, A1, Ap, d, n2, npres, max_levels - 1, max_coarse, steps)
    off0 = field_offsets(n2, npres, d)
    K = [k0["K"]] + Ks
    P0 = _csr(sp.identity(K[0].shape[0], format="csr"))
    P = [P0] + Ps
    field_off = [off0] + offs
    bpat = {0: k0["Bpat"], 1: B1pat}
    patches = [make_patches(K[l], field_off[l], d, Bpattern=bpat[l]) if l in bpat
               else steps.patches(K[l], field_off[l], d) for l in range(len(K) - 1)]
    L = len(K)
    cn = np.zeros(K[-1].shape[0])
    offL = field_off[-1]
    cn[offL[d]:offL[d + 1]] = Bp[L - 2] if L >= 2 else 1.0
    prob = Problem(name=name, dim=d, disc=TH, nu=nu, K=K, P=P, field_off=field_off,
                   patches=patches, b=b, coarse_null=cn,
                   dirichlet=np.concatenate([bnd] * d + [np.zeros(npres, bool)]),
                   Mp=k0["Mp"], exact=exact)
    # diagonal of the P2 velocity mass matrix on every component (DLSC on K0)
    prob.Mu_diag = np.tile(k0["Mu"].diagonal(), d)
    prob.lambda_A, prob.lambda_S = dlsc_bounds(K, field_off, d, mu_diag0=prob.Mu_diag)
    prob.info = dict(mesh=mesh, V=V, n2=n2, npres=npres, Mu=k0["Mu"])
    return prob


def perturb_interior(mesh, amount, seed):
    """Move every interior vertex of a unit-square/cube mesh by independent
    U(-amount, amount) offsets per coordinate (seeded)."""
    s = mesh.scale
    interior = np.all((mesh.key > 0) & (mesh.key < s), axis=1)
    d = mesh.dim
    u = rng.uniform(seed, mesh.nv * d, -amount, amount).reshape(mesh.nv, d)
    x = mesh.x.copy()
    x[interior] += u[interior]
    out = M.Mesh(x, mesh.cells, mesh.key, mesh.scale)
    return out


def build_sv(n, nu=1.0, perturb=0.2, seed_perturb=3001, seed_f=3002, max_levels=10, max_coarse=50,
             name="sv"):
    """Scott-Vogelius P2/P1disc on the Alfeld split R_B of an n x n mesh
    (Sec. 2.1), no-slip walls, f with i.i.d. N(0,1) P2 nodal values per
    component.  K1 is P1isoP2/P1 with P1 velocity on R_U(R_B) and continuous
    P1 pressure on R_B (Sec. 3.1); P0 = blockdiag(I, Pi) where Pi duplicates
    a vertex value into the discontinuous DoFs at that vertex; the pressure
    restriction is R0^p = Mcg^-1 Pi^T M_dg (the L2 projection)."""
    base = M.unit_square(n)
    if perturb:
        base = perturb_interior(base, perturb / n, seed_perturb)
    mesh = M.barycentric_refine(base)
    vol = M.cell_measure(mesh.x, mesh.cells)
    assert vol.min() > 0.0
    d = 2
    V = M.P2Space(mesh)
    n2 = V.n
    nc = mesh.nc
    ndg = 3 * nc
    pdg = np.arange(ndg).reshape(nc, 3)       # P1disc DoF (c, k) = 3c + k
    b2 = fem.p2_basis(d)
    b1 = fem.p1_basis(d)
    A = fem.assemble_stiffness(mesh.x, mesh.cells, V.cell_nodes, fem.stiffness_tensor(b2, d), n2, coef=nu)
    Bs = fem.assemble_div(mesh.x, mesh.cells, pdg, V.cell_nodes, fem.div_tensor(b1, b2, d), ndg, n2)
    bnd = M.p2_boundary_nodes(V)
    uD = [np.zeros(n2), np.zeros(n2)]
    Mu = fem.assemble_mass(mesh.x, mesh.cells, V.cell_nodes, V.cell_nodes, fem.mass_tensor(b2, b2, d), n2, n2)
    z = rng.normal(seed_f, d * n2)
    F = [Mu @ z[c * n2:(c + 1) * n2] for c in range(d)]
    A_in, B_in, F_in, g = dirichlet_eliminate(A, Bs, bnd, uD, F)
    K0 = saddle([A_in] * d, [nonzero_only(B) for B in B_in])
    b = np.concatenate(F_in + [g])
    # transfers and masses
    ncg = mesh.nv
    Pi = _csr(sp.csr_matrix((np.ones(ndg), (pdg.ravel(), mesh.cells.ravel())), shape=(ndg, ncg)))
    Mdg = fem.assemble_mass(mesh.x, mesh.cells, pdg, pdg, fem.mass_tensor(b1, b1, d), ndg, ndg)
    Mcg = fem.assemble_mass(mesh.x, mesh.cells, mesh.cells, mesh.cells, fem.mass_tensor(b1, b1, d), ncg, ncg)
    R0p = _csr(Pi.T @ Mdg)
    # K1 and hierarchy
    K1, A1, B1pat = p1iso_K1(V, mesh.cells, None, ncg, bnd, nu)
    Ap = pressure_laplacian(mesh)
    Ks, Ps, offs, Bp = build_hierarchy(K1, A1, Ap, d, n2, ncg, max_levels - 1, max_coarse)
    off0 = field_offsets(n2, ndg, d)
    K = [K0] + Ks
    P0 = _blockdiag([sp.identity(n2, format="csr")] * d + [Pi])
    P = [P0] + Ps
    field_off = [off0] + offs
    seeds0 = pdg  # three seeds per cell, from the element-to-DoF map (Sec. 3.3.1)
    patches = [make_patches(K[0], off0, d, seeds=seeds0, Bpattern=B_in)]
    bpat = {1: B1pat}
    patches += [make_patches(K[l], field_off[l], d, Bpattern=bpat.get(l)) for l in range(1, len(K) - 1)]
    L = len(K)
    cn = np.zeros(K[-1].shape[0])
    offL = field_off[-1]
    cn[offL[d]:offL[d + 1]] = Bp[L - 2] if L >= 2 else 1.0
    prob = Problem(name=name, dim=d, disc=SV, nu=nu, K=K, P=P, field_off=field_off, patches=patches, b=b,
                   coarse_null=cn, dirichlet=np.concatenate([bnd] * d + [np.zeros(ndg, bool)]),
                   Mp=Mdg, R0p=R0p, Mcg=Mcg, mcg_bounds=(0.5, 2.0))
    prob.lambda_A, prob.lambda_S = dlsc_bounds(K, field_off, d)
    prob.info = dict(mesh=mesh, base=base, V=V, n2=n2, npres=ndg, Mu=Mu, Mdg=Mdg, Pi=Pi)
    return prob


def divergence_norm(prob, x):
    """|| div u_h ||_L2 of the velocity part of x for a P2/P1disc problem:
    B u = -M_dg div_h u, so ||div u_h||^2 = (B u)^T M_dg^-1 (B u)."""
    off = prob.field_off[0]
    d = prob.dim
    K = prob.K[0]
    Bu = K[off[d]:off[d + 1], : off[d]] @ x[: off[d]]
    Mdg = prob.info["Mdg"].tocsc()
    import scipy.sparse.linalg as spla
    w = spla.spsolve(Mdg, Bu)
    return float(np.sqrt(max(Bu @ w, 0.0)))
