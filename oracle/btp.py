"""The block-triangular (inexact Uzawa) comparison preconditioner BTP of
Sec. 4, FP64 (test infrastructure: only tests, the smoke check and the
benchmark's CPU baseline use it).

With [r_u, r_p] = b - K x the update is
    du = Q_A^-1 r_u,        dp = Q_B^-1 (B du - r_p),
the lower block-triangular factor of K = [A B^T; B 0] with the Schur
complement replaced by Q_B.  Q_A^-1 is one SA V-cycle on the vector
Laplacian whose relaxation is two steps of Krylov-wrapped Jacobi (pre and
post) and whose coarsest level is solved exactly; Q_B^-1 is the same kind
of V-cycle on M_p / nu (Taylor-Hood) or the exact block-diagonal inverse
(Scott-Vogelius).

Readings: the V-cycle runs from a zero guess; Dirichlet velocity rows are
identity rows of A, decoupled, so du takes r_u there exactly (as the DC
cycle does).
"""
import numpy as np
import scipy.linalg as sla

from .cycle import krylov_relax


class SAVCycle:
    """One V-cycle of a Galerkin SA hierarchy: `steps` Krylov-wrapped Jacobi
    steps before and after the coarse correction, exact coarsest solve."""

    def __init__(self, As, Ps, steps=2):
        self.A = [a.tocsr() for a in As]
        self.P = [p.tocsr() for p in Ps]
        self.dinv = [1.0 / a.diagonal() for a in self.A]
        self.steps = steps
        self.lu = sla.lu_factor(self.A[-1].toarray())

    def _cycle(self, l, b):
        if l == len(self.A) - 1:
            return sla.lu_solve(self.lu, b)
        A, dinv = self.A[l], self.dinv[l]
        x = krylov_relax(A, np.zeros_like(b), b, lambda v: dinv * v, self.steps)
        e = self._cycle(l + 1, self.P[l].T @ (b - A @ x))
        x = x + self.P[l] @ e
        return krylov_relax(A, x, b, lambda v: dinv * v, self.steps)

    def apply(self, b):
        return self._cycle(0, np.asarray(b, dtype=np.float64))


class BTPOracle:
    def __init__(self, btp, steps=2):
        self.bt = btp
        self.nu = btp.A[0].shape[0]
        self.QA = SAVCycle(btp.A, btp.PA, steps)
        self.QB = SAVCycle(btp.M, btp.PM, steps) if btp.Minv is None else None
        self.B = btp.B.tocsr()
        self.dir = btp.dirichlet_u

    def apply(self, r):
        r = np.asarray(r, dtype=np.float64)
        ru, rp = r[:self.nu], r[self.nu:]
        du = self.QA.apply(ru)
        du[self.dir] = ru[self.dir]
        t = self.B @ du - rp
        dp = self.QB.apply(t) if self.QB is not None else self.bt.Minv @ t
        return np.concatenate([du, dp])
