"""L2 errors of P2 / P1 finite-element functions against exact fields, by a
collapsed (Duffy) tensor Gauss-Legendre rule on each triangle."""
import numpy as np

from problems import fem


def duffy_rule(npts=6):
    t, w = np.polynomial.legendre.leggauss(npts)
    t = 0.5 * (t + 1.0)
    w = 0.5 * w
    U, Vv = np.meshgrid(t, t, indexing="ij")
    WU, WV = np.meshgrid(w, w, indexing="ij")
    s = U.ravel()
    tt = (Vv * (1.0 - U)).ravel()
    wt = (WU * WV * (1.0 - U)).ravel() * 2.0  # reference area 1/2 -> factor 2|T|
    lam = np.stack([1.0 - s - tt, s, tt], axis=1)
    return lam, wt


def l2_error(x, cells, dofs, basis, coef, exact):
    """|| sum_j coef_j phi_j - exact ||_L2 over the triangles ``cells``."""
    lam, wt = duffy_rule()
    vol, _ = fem.geometry(x, cells)
    phi = fem.eval_basis(basis, lam)             # nq x nb
    X = np.einsum("qk,ckd->cqd", lam, x[cells])  # physical points
    uh = np.einsum("qb,cb->cq", phi, coef[dofs])
    ue = exact(X.reshape(-1, 2)).reshape(uh.shape)
    return np.sqrt(np.sum(vol[:, None] * wt[None, :] * (uh - ue) ** 2) / 1.0)
