"""Scalar smoothed-aggregation AMG setup, applied field by field as in
Alg. 1 (Sec. 3.2): strength of connection, greedy aggregation, tentative
prolongator carrying the near-null vector, Jacobi prolongator smoothing and
Galerkin coarse operators.

Readings (the paper defers to PyAMG for these steps):
* strength: the symmetric measure |a_ij| > theta sqrt(|a_ii a_jj|), theta = 0
  (the paper uses the evolution measure, Sec. 3.2; the symmetric one coarsens
  the structured problems here at matched rates);
* aggregation: Vanek-Mandel-Brezina greedy aggregation in natural order;
* smoothing: P = (I - (4/3) / rho(D^-1 A) D^-1 A) T, rho from 30 Lanczos
  steps with a seeded start vector;
* rows with no off-diagonal entries (Dirichlet identity rows) are left out of
  every aggregate, so their rows of P are zero.
"""
import numpy as np
import scipy.sparse as sp

from . import rng


def strength(A, theta=0.0):
    A = A.tocsr()
    d = np.abs(A.diagonal())
    r = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    c = A.indices
    v = np.abs(A.data)
    keep = (r != c) & (v > theta * np.sqrt(d[r] * d[c]))
    S = sp.csr_matrix((np.ones(keep.sum()), (r[keep], c[keep])), shape=A.shape)
    S.sort_indices()
    return S


def aggregate(S, excluded):
    """Greedy aggregation.  Returns agg (n,) with -1 for excluded nodes and the
    number of aggregates.

    Pass 1: a node whose strong neighbours are all free starts an aggregate
    with them.  Pass 2: each remaining free node joins the aggregate of its
    first strong neighbour aggregated in pass 1.  Pass 3: each still-free node
    starts an aggregate with its free strong neighbours."""
    n = S.shape[0]
    ptr = S.indptr.tolist()
    idx = S.indices.tolist()
    agg = [-1] * n
    excl = excluded.tolist()
    na = 0
    for i in range(n):
        if excl[i] or agg[i] >= 0:
            continue
        nb = idx[ptr[i]:ptr[i + 1]]
        if all(agg[j] < 0 for j in nb):
            agg[i] = na
            for j in nb:
                agg[j] = na
            na += 1
    snap = list(agg)
    for i in range(n):
        if excl[i] or agg[i] >= 0:
            continue
        for j in idx[ptr[i]:ptr[i + 1]]:
            if snap[j] >= 0:
                agg[i] = snap[j]
                break
    for i in range(n):
        if excl[i] or agg[i] >= 0:
            continue
        agg[i] = na
        for j in idx[ptr[i]:ptr[i + 1]]:
            if agg[j] < 0 and not excl[j]:
                agg[j] = na
        na += 1
    return np.array(agg, dtype=np.int64), na


def tentative(agg, na, B):
    """Columns of T are the near-null vector B restricted to an aggregate and
    normalised; Bc holds the norms, so that T Bc = B on aggregated rows."""
    n = agg.size
    rows = np.nonzero(agg >= 0)[0]
    cols = agg[rows]
    nrm = np.sqrt(np.bincount(cols, weights=B[rows] ** 2, minlength=na))
    T = sp.csr_matrix((B[rows] / nrm[cols], (rows, cols)), shape=(n, na))
    T.sort_indices()
    return T, nrm


def lanczos_max(A, steps=30, seed=12345):
    """Largest eigenvalue estimate of a symmetric operator by Lanczos with
    full reorthogonalisation and a seeded start vector."""
    n = A.shape[0]
    steps = min(steps, n)
    v = rng.uniform(seed, n, -1.0, 1.0)
    v /= np.linalg.norm(v)
    V = np.zeros((steps + 1, n))
    V[0] = v
    a = np.zeros(steps)
    b = np.zeros(steps)
    k_used = steps
    for k in range(steps):
        w = A @ V[k]
        a[k] = w @ V[k]
        w -= V[: k + 1].T @ (V[: k + 1] @ w)
        w -= V[: k + 1].T @ (V[: k + 1] @ w)
        b[k] = np.linalg.norm(w)
        if b[k] < 1e-12 * max(1.0, abs(a[k])):
            k_used = k + 1
            break
        V[k + 1] = w / b[k]
    T = np.diag(a[:k_used]) + np.diag(b[: k_used - 1], 1) + np.diag(b[: k_used - 1], -1)
    return float(np.linalg.eigvalsh(T).max())


def rho_DinvA(A, mask):
    """Spectral radius estimate of D^-1 A restricted to the rows in mask."""
    idx = np.nonzero(mask)[0]
    As = A[idx][:, idx]
    dis = 1.0 / np.sqrt(As.diagonal())
    M = sp.diags(dis) @ As @ sp.diags(dis)
    return lanczos_max(M.tocsr())


def smooth_prolongator(A, T, excluded):
    mask = ~excluded
    rho = rho_DinvA(A, mask)
    omega = (4.0 / 3.0) / rho
    dinv = np.zeros(A.shape[0])
    dinv[mask] = 1.0 / A.diagonal()[mask]
    P = T - omega * (sp.diags(dinv) @ (A @ T))
    P = sp.csr_matrix(P)
    P.eliminate_zeros()
    P.sort_indices()
    return P


def isolated_rows(A):
    """Rows whose only stored entry is the diagonal (Dirichlet identity rows)."""
    A = A.tocsr()
    r = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    off = (A.indices != r) & (A.data != 0)
    return np.bincount(r[off], minlength=A.shape[0]) == 0


def sa_field(A, B, max_levels, max_coarse=50, theta=0.0):
    """Scalar SA hierarchy for one field: returns lists Ps, As, Bs, where
    As[0] = A and Ps[k] maps level k+1 to level k.  Coarsening stops when the
    field has at most max_coarse DoFs or max_levels levels exist."""
    As, Ps, Bs = [A.tocsr()], [], [B]
    while len(As) < max_levels and As[-1].shape[0] > max_coarse:
        Ak = As[-1]
        excl = isolated_rows(Ak)
        S = strength(Ak, theta)
        agg, na = aggregate(S, excl)
        if na == 0 or na >= Ak.shape[0]:
            break
        T, Bc = tentative(agg, na, Bs[-1])
        P = smooth_prolongator(Ak, T, excl)
        Ac = (P.T @ Ak @ P).tocsr()
        Ac.sort_indices()
        Ps.append(P)
        As.append(Ac)
        Bs.append(Bc)
    return Ps, As, Bs
