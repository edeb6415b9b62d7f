"""DLSC relaxation, FP64 (Sec. 3.3.2, Alg. 2).

One sweep for [A B^T; B 0] [u; p] = [f; g] with the velocity mass matrix
replaced by Mu: its diagonal on the P2/P1 grid (level 0, K0), the identity
on the P1isoP2 hierarchy (levels >= 1), as Sec. 3.3.2 prescribes:

    v* ~ A^-1 (f - A u - B^T p)                   (momentum)
    q  ~ (B Mu^-1 B^T)^-1 (g - B (u + v*))         (continuity)
    dp ~ (B Mu^-1 B^T)^-1 ( -(B Mu^-1 A Mu^-1 B^T) q )   (pressure correction)
    du = v* + Mu^-1 B^T q
    u += du,  p += dp

Each approximate solve is a Chebyshev semi-iteration from a zero guess on
the interval [0.5^d lam, 1.1 lam], lam the largest-eigenvalue estimate of A
or of B Mu^-1 B^T (Table lsd_dgs_config), with the stage's degree.
Reading: the pressure-correction right-hand side carries the minus sign of
the derivation (A_p-hat enters the factorisation with a minus); the displayed
iteration (Eq. fulldlsc) shows a plus.
"""
import numpy as np


def chebyshev(op, b, lo, hi, degree, dinv=None):
    """x ~= A^-1 b by `degree` steps of the Chebyshev semi-iteration for
    eigenvalues of (D^-1) A in [lo, hi], zero initial guess (Saad,
    Iterative Methods for Sparse Linear Systems, Alg. 12.1)."""
    theta = 0.5 * (hi + lo)
    delta = 0.5 * (hi - lo)
    sigma = theta / delta
    rho = 1.0 / sigma
    x = np.zeros_like(b)
    r = b.copy() if dinv is None else dinv * b
    d = r / theta
    for _ in range(degree):
        x = x + d
        Ad = op(d)
        r = r - (Ad if dinv is None else dinv * Ad)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + 2.0 * rho_new / delta * r
        rho = rho_new
    return x


class DLSCLevel:
    """DLSC data of level l.  Mu^-1 is 1 / prob.Mu_diag on level 0 (the
    high-order P2 grid) and the identity on levels >= 1 (P1isoP2 grids);
    lambda_S[l] is the largest-eigenvalue estimate of B Mu^-1 B^T."""

    def __init__(self, prob, l, params):
        K = prob.K[l].tocsr()
        off = prob.field_off[l]
        d = prob.dim
        nv = off[d]
        self.nv = nv
        self.K = K
        self.A = K[:nv, :nv].tocsr()
        self.B = K[nv:, :nv].tocsr()
        self.BT = K[:nv, nv:].tocsr()
        if l == 0:
            if getattr(prob, "Mu_diag", None) is None:
                raise ValueError("DLSC on level 0 needs the velocity mass diagonal Mu_diag")
            self.mu_inv = 1.0 / np.asarray(prob.Mu_diag, dtype=np.float64)
            assert self.mu_inv.size == nv
        else:
            self.mu_inv = np.ones(nv)
        self.dim = d
        self.lamA = float(prob.lambda_A[l])
        self.lamS = float(prob.lambda_S[l])
        self.deg = tuple(params.cheb_deg)
        self.sweeps = params.dlsc_sweeps

    def one(self, x, rhs):
        nv = self.nv
        mi = self.mu_inv
        u, p = x[:nv], x[nv:]
        f, g = rhs[:nv], rhs[nv:]
        sA = (0.5 ** self.dim * self.lamA, 1.1 * self.lamA)
        sS = (0.5 ** self.dim * self.lamS, 1.1 * self.lamS)
        S = lambda y: self.B @ (mi * (self.BT @ y))
        # momentum, continuity, pressure correction, velocity correction
        v = chebyshev(lambda y: self.A @ y, f - self.A @ u - self.BT @ p, sA[0], sA[1], self.deg[0])
        q = chebyshev(S, g - self.B @ (u + v), sS[0], sS[1], self.deg[1])
        dp = chebyshev(S, -(self.B @ (mi * (self.A @ (mi * (self.BT @ q))))), sS[0], sS[1], self.deg[2])
        du = v + mi * (self.BT @ q)
        return np.concatenate([u + du, p + dp])

    def sweep(self, x, b):
        for _ in range(self.sweeps):
            x = self.one(x, b)
        return x
