"""Simplicial meshes of the unit square and cube, their refinements, and the
P2 / P1disc node numberings used by the Stokes problems.

* ``unit_square(n)``: n x n squares, each split along the diagonal from
  (x, y) to (x+h, y+h) (the "right" diagonal) into two triangles.
* ``unit_cube(n)``: n^3 cubes, each split into 6 tetrahedra sharing the main
  diagonal (Freudenthal / Kuhn split).
* ``barycentric_refine``: the Alfeld split R_B of Sec. 2.1 (each triangle
  becomes three around its centroid).
* ``uniform_refine``: the quadrisection R_U of Sec. 2.1 in 2D (four children
  through the edge midpoints) and the red 1->8 split in 3D (Bey's ordering,
  which keeps Kuhn congruence; the paper is silent on the 3D diagonal).

Nodes are ordered lexicographically by (z, y, x) of their unperturbed
positions so that matrices are banded and gathers are local.
"""
import numpy as np

# Local edges of a cell, in the order used for P2 edge nodes.
EDGES = {2: np.array([[0, 1], [1, 2], [0, 2]]),
         3: np.array([[0, 1], [0, 2], [0, 3], [1, 2], [1, 3], [2, 3]])}


class Mesh:
    """Vertices ``x`` (nv x d), cells ``cells`` (nc x (d+1)).

    ``key`` holds integer lattice coordinates of the unperturbed vertices
    (used only for ordering and boundary detection); ``scale`` converts them
    back to coordinates (x_unperturbed = key / scale).
    """

    def __init__(self, x, cells, key, scale):
        self.x = np.asarray(x, dtype=np.float64)
        self.cells = np.asarray(cells, dtype=np.int64)
        self.key = np.asarray(key, dtype=np.int64)
        self.scale = int(scale)

    @property
    def dim(self):
        return self.x.shape[1]

    @property
    def nv(self):
        return self.x.shape[0]

    @property
    def nc(self):
        return self.cells.shape[0]


def _lex_order(key):
    # sort by last coordinate first (z, then y, then x)
    return np.lexsort(tuple(key[:, k] for k in range(key.shape[1])))


def _renumber(mesh_x, cells, key, scale):
    order = _lex_order(key)
    inv = np.empty_like(order)
    inv[order] = np.arange(order.size)
    return Mesh(mesh_x[order], inv[cells], key[order], scale)


def unit_square(n):
    """n x n squares, each split by the (x,y)-(x+h,y+h) diagonal."""
    i, j = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="xy")
    key = np.stack([i.ravel(), j.ravel()], axis=1)  # vertex id = j*(n+1)+i
    x = key / n
    v = lambda a, b: b * (n + 1) + a
    a, b = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    a = a.ravel(); b = b.ravel()
    v00, v10, v11, v01 = v(a, b), v(a + 1, b), v(a + 1, b + 1), v(a, b + 1)
    lower = np.stack([v00, v10, v11], axis=1)
    upper = np.stack([v00, v11, v01], axis=1)
    cells = np.stack([lower, upper], axis=1).reshape(-1, 3)
    return Mesh(x, cells, key, n)


def unit_cube(n):
    """n^3 cubes, each split into 6 tetrahedra along the (0,0,0)-(1,1,1) diagonal."""
    g = np.arange(n + 1)
    i, j, k = np.meshgrid(g, g, g, indexing="ij")
    key = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)
    vid = lambda a, b, c: (a * (n + 1) + b) * (n + 1) + c
    x = key / n
    a, b, c = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    a = a.ravel(); b = b.ravel(); c = c.ravel()
    cells = []
    # Kuhn simplices: paths from (0,0,0) to (1,1,1) along the 6 axis orders
    for perm in ([0, 1, 2], [0, 2, 1], [1, 0, 2], [1, 2, 0], [2, 0, 1], [2, 1, 0]):
        p = [np.zeros_like(a)] * 3
        cur = [a.copy(), b.copy(), c.copy()]
        verts = [vid(*cur)]
        for ax in perm:
            cur = list(cur)
            cur[ax] = cur[ax] + 1
            verts.append(vid(*cur))
        cells.append(np.stack(verts, axis=1))
    cells = np.stack(cells, axis=1).reshape(-1, 4)
    return _renumber(x, cells, key, n)


def cell_measure(x, cells):
    """Signed-free volume |T| of each simplex."""
    d = x.shape[1]
    J = x[cells[:, 1:]] - x[cells[:, :1]]  # nc x d x d (rows = edge vectors)
    det = np.linalg.det(J)
    return np.abs(det) / (2.0 if d == 2 else 6.0)


def edges_of(mesh):
    """Unique edges (ne x 2, sorted endpoints) and the cell->edge map."""
    d = mesh.dim
    le = EDGES[d]
    e = np.sort(mesh.cells[:, le], axis=2).reshape(-1, 2)
    uniq, inv = np.unique(e, axis=0, return_inverse=True)
    return uniq, inv.reshape(mesh.nc, le.shape[0])


class P2Space:
    """P2 nodes of a mesh: vertices plus edge midpoints, renumbered
    lexicographically.  ``cell_nodes`` (nc x nb) lists each cell's nodes in
    local order (vertices, then edges in ``EDGES`` order); ``vert_node`` maps a
    mesh vertex to its node number."""

    def __init__(self, mesh):
        d = mesh.dim
        edges, c2e = edges_of(mesh)
        nv = mesh.nv
        key = np.concatenate([2 * mesh.key, mesh.key[edges[:, 0]] + mesh.key[edges[:, 1]]])
        x = np.concatenate([mesh.x, 0.5 * (mesh.x[edges[:, 0]] + mesh.x[edges[:, 1]])])
        order = _lex_order(key)
        inv = np.empty_like(order)
        inv[order] = np.arange(order.size)
        raw = np.concatenate([mesh.cells, nv + c2e], axis=1)
        self.mesh = mesh
        self.x = x[order]
        self.key = key[order]
        self.scale = 2 * mesh.scale
        self.cell_nodes = inv[raw]
        self.vert_node = inv[:nv]
        self.edges = edges
        self.edge_node = inv[nv:]
        self.n = x.shape[0]


def boundary_facets(mesh):
    """Facets (edges in 2D, triangles in 3D) that belong to exactly one cell."""
    d = mesh.dim
    faces = []
    for k in range(d + 1):
        faces.append(np.delete(mesh.cells, k, axis=1))
    f = np.sort(np.concatenate(faces), axis=1)
    uniq, cnt = np.unique(f, axis=0, return_counts=True)
    return uniq[cnt == 1]


def p2_boundary_nodes(space):
    """Boolean mask of P2 nodes lying on the domain boundary."""
    mesh = space.mesh
    bf = boundary_facets(mesh)
    mask = np.zeros(space.n, dtype=bool)
    mask[space.vert_node[bf.ravel()]] = True
    # edge nodes of boundary facets
    d = mesh.dim
    ek = {tuple(e): i for i, e in enumerate(map(tuple, space.edges))} if False else None
    e_sorted = space.edges
    # boundary edges = all edges of boundary facets
    if d == 2:
        be = np.sort(bf, axis=1)
    else:
        be = np.sort(np.concatenate([bf[:, [0, 1]], bf[:, [1, 2]], bf[:, [0, 2]]]), axis=1)
    be = np.unique(be, axis=0)
    # locate be in e_sorted
    ne = e_sorted.shape[0]
    code_all = e_sorted[:, 0] * (mesh.nv + 1) + e_sorted[:, 1]
    code_b = be[:, 0] * (mesh.nv + 1) + be[:, 1]
    pos = np.searchsorted(code_all, code_b)
    assert np.all(code_all[pos] == code_b)
    mask[space.edge_node[pos]] = True
    return mask


def barycentric_refine(mesh):
    """Alfeld split R_B: add each triangle's centroid and split it into 3.
    Children of a cell are stored consecutively, in parent order; the
    centroid is the last vertex of each child."""
    assert mesh.dim == 2
    nv, nc = mesh.nv, mesh.nc
    cx = mesh.x[mesh.cells].mean(axis=1)
    ckey = mesh.key[mesh.cells].sum(axis=1)  # 3 * centroid lattice coords
    key = np.concatenate([3 * mesh.key, ckey])
    x = np.concatenate([mesh.x, cx])
    c = mesh.cells
    m = nv + np.arange(nc)
    ch = np.stack([np.stack([c[:, 0], c[:, 1], m], 1),
                   np.stack([c[:, 1], c[:, 2], m], 1),
                   np.stack([c[:, 2], c[:, 0], m], 1)], axis=1).reshape(-1, 3)
    order = _lex_order(key)
    inv = np.empty_like(order)
    inv[order] = np.arange(order.size)
    out = Mesh(x[order], inv[ch], key[order], 3 * mesh.scale)
    out.parent = np.repeat(np.arange(nc), 3)
    return out


# Children of the reference simplex under uniform refinement, as lists of
# local P2 node indices (vertices 0..d, then edges in EDGES order).
def _children(d):
    if d == 2:
        # nodes: 0,1,2 vertices; 3=(0,1) 4=(1,2) 5=(0,2)
        return np.array([[0, 3, 5], [3, 1, 4], [5, 4, 2], [3, 4, 5]])
    # 3D: nodes 0..3 vertices; 4=(0,1) 5=(0,2) 6=(0,3) 7=(1,2) 8=(1,3) 9=(2,3)
    # Bey's red refinement: 4 corner tets and 4 tets around the (0,2)-(1,3)
    # edge... using the fixed local ordering x0, x01, x02, x03 etc.
    m01, m02, m03, m12, m13, m23 = 4, 5, 6, 7, 8, 9
    return np.array([
        [0, m01, m02, m03],
        [m01, 1, m12, m13],
        [m02, m12, 2, m23],
        [m03, m13, m23, 3],
        [m01, m02, m03, m13],
        [m01, m02, m12, m13],
        [m02, m03, m13, m23],
        [m02, m12, m13, m23],
    ])


CHILDREN = {2: _children(2), 3: _children(3)}


def child_barycentrics(d):
    """Parent barycentric coordinates of every local P2 node ((d+1)+ne x (d+1))."""
    nb = d + 1
    pts = [np.eye(nb)[i] for i in range(nb)]
    for a, b in EDGES[d]:
        pts.append(0.5 * (np.eye(nb)[a] + np.eye(nb)[b]))
    return np.array(pts)


def uniform_refine_cells(space):
    """Cells of R_U(mesh) on the P2 node numbering of ``space`` (children of
    cell c are rows 2^d*c .. 2^d*c+2^d-1), plus the parent-barycentric
    coordinates of each child's vertices (2^d x (d+1) x (d+1))."""
    d = space.mesh.dim
    ch = CHILDREN[d]
    cells = space.cell_nodes[:, ch].reshape(-1, d + 1)
    bary = child_barycentrics(d)[ch]
    return cells, bary
