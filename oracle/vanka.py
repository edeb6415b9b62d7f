"""Additive Vanka relaxation (Sec. 3.3.1).

One sweep on level l is x <- x + omega * M^-1 (b - K x) with

    M^-1 = sum_i V_i^T W_i (V_i K V_i^T)^-1 V_i          (Eq. vanka)

V_i injects the DoFs of patch i, W_i is the partition of unity whose entries
are 1 / (number of patches holding the DoF).  Each patch system
K_i = V_i K V_i^T is formed densely and solved by LU with partial pivoting
(LAPACK gesv) - deliberately not the block factorisation of Eqs.
vanka_fact1/2 that the CUDA path uses.
"""
import numpy as np


def patch_lists(patches):
    ptr, dof = patches.ptr, patches.dof
    return [dof[ptr[i]:ptr[i + 1]] for i in range(ptr.size - 1)]


def partition_of_unity(patches, n):
    """Diagonal of W: 1 / number of patches holding each DoF (0 if none)."""
    cnt = np.bincount(patches.dof, minlength=n).astype(np.float64)
    w = np.zeros(n)
    w[cnt > 0] = 1.0 / cnt[cnt > 0]
    return w


class VankaLevel:
    """Dense patch matrices K_i = V_i K V_i^T of one level, grouped by size
    so that numpy can solve each group in one call (the solves are
    independent, so grouping changes no result)."""

    def __init__(self, K, patches):
        K = K.tocsr()
        K.sort_indices()
        self.n = K.shape[0]
        self.W = partition_of_unity(patches, self.n)
        lists = patch_lists(patches)
        sizes = np.array([len(p) for p in lists])
        self.groups = []
        for m in np.unique(sizes):
            ids = np.nonzero(sizes == m)[0]
            idx = np.stack([lists[i] for i in ids]).astype(np.int64)  # g x m
            mats = np.concatenate([self._dense_blocks(K, idx[s:s + 4096]) for s in range(0, len(ids), 4096)])
            self.groups.append((ids, idx, mats))
        self.npatch = len(lists)

    @staticmethod
    def _dense_blocks(K, idx):
        """K_i = V_i K V_i^T for a batch of equal-size patches (rows of idx):
        entry (a, b) of patch i is K[idx[i, a], idx[i, b]] (0 if not stored)."""
        g, m = idx.shape
        assert np.all(np.diff(idx, axis=1) > 0), "patch lists ascend (velocity x, y[, z], pressure)"
        out = np.zeros((g, m, m))
        rows = idx.ravel()
        cnt = np.diff(K.indptr)[rows]
        pid = np.repeat(np.arange(g * m), cnt)              # (patch, local row) of each entry
        starts = np.repeat(K.indptr[rows], cnt)
        offs = np.arange(cnt.sum()) - np.repeat(np.cumsum(cnt) - cnt, cnt)
        cols = K.indices[starts + offs]
        vals = K.data[starts + offs]
        p = pid // m
        a = pid % m
        # local column: position of cols in the patch list (ascending, exact match)
        key_tab = (np.arange(g)[:, None] * (K.shape[1] + 1) + idx).ravel()   # sorted: lists ascend
        key = p * (K.shape[1] + 1) + cols
        pos = np.searchsorted(key_tab, key)
        pos = np.minimum(pos, key_tab.size - 1)
        hit = key_tab[pos] == key
        b = pos - p * m
        out[p[hit], a[hit], b[hit]] = vals[hit]
        return out

    def apply(self, r):
        """Return M^-1 r = sum_i V_i^T W_i K_i^-1 V_i r, summing each DoF's
        contributions in ascending patch order."""
        ixs = [None] * self.npatch
        ys = [None] * self.npatch
        for ids, idx, mats in self.groups:
            y = np.linalg.solve(mats, r[idx][:, :, None])[:, :, 0]
            for k, i in enumerate(ids):
                ixs[i] = idx[k]
                ys[i] = y[k]
        acc = np.zeros(self.n)
        if self.npatch:
            # np.add.at accumulates sequentially, i.e. in ascending patch order
            np.add.at(acc, np.concatenate(ixs), np.concatenate(ys))
        return self.W * acc

    def sweep(self, K, x, b, omega):
        """One stationary damped sweep x <- x + omega M^-1 (b - K x)."""
        return x + omega * self.apply(b - K @ x)


def sampled_apply(K, patches, r, dofs):
    """(M^-1 r)[dofs] of Eq. vanka computed from only the patches that hold
    the sampled DoFs, each by a dense LU solve: a check of a full-size Vanka
    application at a handful of entries."""
    K = K.tocsr()
    lists = patch_lists(patches)
    W = partition_of_unity(patches, K.shape[0])
    want = {int(d): 0.0 for d in dofs}
    for ix in lists:
        hit = [int(g) for g in ix if int(g) in want]
        if not hit:
            continue
        y = np.linalg.solve(K[ix][:, ix].toarray(), r[ix])
        pos = {int(g): k for k, g in enumerate(ix)}
        for g in hit:
            want[g] += y[pos[g]]
    return np.array([W[int(d)] * want[int(d)] for d in dofs])
