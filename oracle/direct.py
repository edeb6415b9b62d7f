"""Sparse direct solves of the full Stokes system (pins of the discretisation).

The enclosed-flow system is singular (constant pressure), so it is solved in
bordered form [K n; n^T 0] with n = (0, 1_p), then the pressure is shifted to
zero mass-weighted mean, int p dx = 0 (Sec. 2: pressure in L^2_0)."""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def solve_stokes(K, b, off, dim, Mp=None):
    n = K.shape[0]
    nvec = np.zeros(n)
    nvec[off[dim]:off[dim + 1]] = 1.0
    Kb = sp.bmat([[K, sp.csr_matrix(nvec[:, None])], [sp.csr_matrix(nvec[None, :]), None]], format="csc")
    x = spla.spsolve(Kb, np.concatenate([b, [0.0]]))[:n]
    if Mp is not None:
        x = zero_mean_pressure(x, off, dim, Mp)
    return x


def zero_mean_pressure(x, off, dim, Mp):
    """Shift p so that 1^T Mp p = 0 (mass-weighted mean)."""
    x = x.copy()
    p = x[off[dim]:off[dim + 1]]
    one = np.ones(p.size)
    x[off[dim]:off[dim + 1]] = p - (one @ (Mp @ p)) / (one @ (Mp @ one))
    return x
