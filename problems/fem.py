"""Finite-element assembly for the Stokes problems (Sec. 2, Eq. saddle).

Element integrals are exact: every basis function is a polynomial in the
barycentric coordinates, and integrals of barycentric monomials over a
simplex have the closed form

    int_T l_0^a0 ... l_d^ad dx = |T| d! a0! ... ad! / (d + a0 + ... + ad)!

so no quadrature constants appear.  Bilinear forms (Sec. 2):

    a(u, v) = nu * int grad u : grad v,     b(p, v) = - int p div v.
"""
from math import factorial
from itertools import product

import numpy as np
import scipy.sparse as sp

from .mesh import EDGES


# ---------------------------------------------------------------- polynomials
# A polynomial in barycentric coordinates is a dict {exponent tuple: coeff}.

def _mono(d, k, c=1.0):
    e = [0] * (d + 1)
    e[k] = 1
    return {tuple(e): c}


def _const(d, c):
    return {tuple([0] * (d + 1)): c}


def _add(p, q):
    r = dict(p)
    for e, c in q.items():
        r[e] = r.get(e, 0.0) + c
    return r


def _mul(p, q):
    r = {}
    for (e1, c1), (e2, c2) in product(p.items(), q.items()):
        e = tuple(a + b for a, b in zip(e1, e2))
        r[e] = r.get(e, 0.0) + c1 * c2
    return r


def _scale(p, s):
    return {e: c * s for e, c in p.items()}


def _dlam(p, k):
    """Partial derivative with respect to barycentric coordinate k."""
    r = {}
    for e, c in p.items():
        if e[k] > 0:
            e2 = list(e)
            e2[k] -= 1
            r[tuple(e2)] = r.get(tuple(e2), 0.0) + c * e[k]
    return r


def _integrate(p, d):
    """(1/|T|) * int_T p dx."""
    s = 0.0
    for e, c in p.items():
        num = factorial(d)
        for a in e:
            num *= factorial(a)
        s += c * num / factorial(d + sum(e))
    return s


def p1_basis(d):
    return [_mono(d, k) for k in range(d + 1)]


def p2_basis(d):
    """Vertex functions l_i (2 l_i - 1), then edge functions 4 l_a l_b."""
    out = []
    for i in range(d + 1):
        li = _mono(d, i)
        out.append(_mul(li, _add(_scale(li, 2.0), _const(d, -1.0))))
    for a, b in EDGES[d]:
        out.append(_scale(_mul(_mono(d, a), _mono(d, b)), 4.0))
    return out


def stiffness_tensor(basis, d):
    """C[i, j, k, l] = (1/|T|) int dphi_i/dl_k * dphi_j/dl_l."""
    nb = len(basis)
    C = np.zeros((nb, nb, d + 1, d + 1))
    der = [[_dlam(f, k) for k in range(d + 1)] for f in basis]
    for i, j, k, l in product(range(nb), range(nb), range(d + 1), range(d + 1)):
        C[i, j, k, l] = _integrate(_mul(der[i][k], der[j][l]), d)
    return C


def mass_tensor(b1, b2, d):
    """E[i, j] = (1/|T|) int phi_i psi_j."""
    E = np.zeros((len(b1), len(b2)))
    for i, f in enumerate(b1):
        for j, g in enumerate(b2):
            E[i, j] = _integrate(_mul(f, g), d)
    return E


def div_tensor(pbasis, vbasis, d):
    """D[q, j, k] = (1/|T|) int psi_q * dphi_j/dl_k."""
    D = np.zeros((len(pbasis), len(vbasis), d + 1))
    for q, f in enumerate(pbasis):
        for j, g in enumerate(vbasis):
            for k in range(d + 1):
                D[q, j, k] = _integrate(_mul(f, _dlam(g, k)), d)
    return D


def eval_basis(basis, lam):
    """Values of each basis function at barycentric points lam (np x (d+1))."""
    out = np.zeros((lam.shape[0], len(basis)))
    for i, f in enumerate(basis):
        for e, c in f.items():
            out[:, i] += c * np.prod(lam ** np.array(e), axis=1)
    return out


# ------------------------------------------------------------ geometry
def geometry(x, cells):
    """|T| and barycentric gradients (nc x (d+1) x d) of each simplex."""
    d = x.shape[1]
    X = x[cells]  # nc x (d+1) x d
    J = X[:, 1:, :] - X[:, :1, :]  # rows are edge vectors
    det = np.linalg.det(J)
    vol = np.abs(det) / factorial(d)
    Jinv = np.linalg.inv(J)  # columns give grad of l_1..l_d
    g = np.empty((cells.shape[0], d + 1, d))
    g[:, 1:, :] = np.transpose(Jinv, (0, 2, 1))
    g[:, 0, :] = -g[:, 1:, :].sum(axis=1)
    return vol, g


def _coo(rows, cols, vals, shape, keep_zeros=False):
    """CSR from element contributions.  With keep_zeros the element
    connectivity pattern is kept even where the summed value is zero."""
    m = sp.coo_matrix((vals.ravel(), (rows.ravel(), cols.ravel())), shape=shape).tocsr()
    m.sum_duplicates()
    if not keep_zeros:
        m.eliminate_zeros()
    m.sort_indices()
    return m


def assemble_stiffness(x, cells, dofs, basis_C, n, coef=1.0):
    """Scalar stiffness coef * int grad phi_i . grad phi_j."""
    vol, g = geometry(x, cells)
    G = np.einsum("ckd,cld->ckl", g, g)
    Ke = coef * vol[:, None, None] * np.einsum("ijkl,ckl->cij", basis_C, G)
    nb = dofs.shape[1]
    r = np.repeat(dofs, nb, axis=1)
    c = np.tile(dofs, (1, nb))
    return _coo(r, c, Ke.reshape(len(cells), -1), (n, n))


def assemble_mass(x, cells, rdofs, cdofs, E, nr, nc):
    vol, _ = geometry(x, cells)
    Me = vol[:, None, None] * E[None]
    nbr, nbc = rdofs.shape[1], cdofs.shape[1]
    r = np.repeat(rdofs, nbc, axis=1)
    c = np.tile(cdofs, (1, nbr))
    return _coo(r, c, Me.reshape(len(cells), -1), (nr, nc))


def assemble_div(x, cells, pdofs, vdofs, D, npres, nvel):
    """Per component c: B_c[q, j] = - int psi_q dphi_j/dx_c.  The element
    connectivity pattern is kept (explicit zeros included)."""
    vol, g = geometry(x, cells)
    d = x.shape[1]
    out = []
    npb, nvb = pdofs.shape[1], vdofs.shape[1]
    r = np.repeat(pdofs, nvb, axis=1)
    cc = np.tile(vdofs, (1, npb))
    for comp in range(d):
        Be = -vol[:, None, None] * np.einsum("qjk,ck->cqj", D, g[:, :, comp])
        out.append(_coo(r, cc, Be.reshape(len(cells), -1), (npres, nvel), keep_zeros=True))
    return out
