"""Setup of the block-triangular comparison preconditioner BTP (Sec. 4):
the hierarchies its two approximate inverses run on.

* Q_A: one smoothed-aggregation V-cycle on the vector Laplacian A (the
  velocity block of K0, Dirichlet identity rows included): scalar SA on
  each velocity component's block (Alg. 1's field-by-field setup, the same
  strength/aggregation/smoothing readings), block-diagonal prolongators and
  Galerkin coarse operators.
* Q_B: the pressure-mass matrix scaled by 1/nu (the Schur complement
  B A^-1 B^T is spectrally equivalent to M_p / nu): for Taylor-Hood an SA
  V-cycle on it; for Scott-Vogelius (P1disc, block diagonal per cell) its
  exact inverse, stored as a block-diagonal CSR.

Host setup only: no solve-phase arithmetic.
"""
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import sa
from .stokes import SV, TH


def _csr(m):
    m = sp.csr_matrix(m)
    m.sort_indices()
    return m


@dataclass
class BTPData:
    A: list          # A[l]: velocity operator on level l (A[0] = velocity block of K0)
    PA: list         # PA[l] maps level l+1 to l
    B: sp.csr_matrix  # pressure rows x velocity columns of K0
    M: list          # TH: Q_B hierarchy (M[0] = M_p / nu); SV: []
    PM: list
    Minv: sp.csr_matrix  # SV: exact block-diagonal inverse of M_p / nu; TH: None
    dirichlet_u: np.ndarray


def _vector_hierarchy(A, d, max_levels, max_coarse):
    n2 = A.shape[0] // d
    blocks = [A[c * n2:(c + 1) * n2, c * n2:(c + 1) * n2] for c in range(d)]
    co = A.tocoo()
    cross = (co.row // n2) != (co.col // n2)
    assert not np.any(co.data[cross] != 0.0), "the velocity block couples components"
    hs = [sa.sa_field(Bk, np.ones(n2), max_levels, max_coarse) for Bk in blocks]
    nl = min(len(h[1]) for h in hs)
    As = [_csr(A)]
    Ps = []
    for l in range(nl - 1):
        P = _csr(sp.block_diag([h[0][l] for h in hs], format="csr"))
        Ps.append(P)
        As.append(_csr(P.T @ As[-1] @ P))
    return As, Ps


def _cell_blocks_inverse(M):
    """Exact inverse of a block-diagonal matrix (connected components of its
    pattern are the blocks)."""
    n = M.shape[0]
    ncomp, lab = sp.csgraph.connected_components(M, directed=False)
    rows, cols, vals = [], [], []
    Md = M.tocsr()
    for k in range(ncomp):
        idx = np.nonzero(lab == k)[0]
        blk = Md[idx][:, idx].toarray()
        inv = np.linalg.inv(blk)
        r, c = np.meshgrid(idx, idx, indexing="ij")
        rows.append(r.ravel())
        cols.append(c.ravel())
        vals.append(inv.ravel())
    return _csr(sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n)))


def build_btp(prob, max_levels=10, max_coarse=50):
    d = prob.dim
    off = prob.field_off[0]
    nu_ = off[d]
    K = prob.K[0].tocsr()
    A = _csr(K[:nu_, :nu_])
    B = _csr(K[nu_:, :nu_])
    As, Ps = _vector_hierarchy(A, d, max_levels, max_coarse)
    Q = _csr(prob.Mp / prob.nu)
    if prob.disc == TH:
        Pm, Ms, _ = sa.sa_field(Q, np.ones(Q.shape[0]), max_levels, max_coarse)
        return BTPData(A=As, PA=Ps, B=B, M=Ms, PM=Pm, Minv=None, dirichlet_u=prob.dirichlet[:nu_].copy())
    assert prob.disc == SV
    return BTPData(A=As, PA=Ps, B=B, M=[], PM=[], Minv=_cell_blocks_inverse(Q),
                   dirichlet_u=prob.dirichlet[:nu_].copy())
