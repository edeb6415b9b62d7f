"""The defect-correction (DC) preconditioner, FP64 (Sec. 3.1 and 3.2).

Error propagation of one application (Eq. TG-operator-full, gamma = 1):

    G_dc = (I - w0 M0^-1 K0)^nu2 (I - P0 (I - G1) K1^-1 eta R0 K0) (I - w0 M0^-1 K0)^nu1

Applied to a residual r with a zero initial guess:

    1. nu1 relaxation sweeps on K0;
    2. d = eta (r - K0 x), eta = diag(eta_u I, eta_p I)       (Eq. eta)
    3. d1 = R0 d                                              (Eq. interp)
    4. e = one V-cycle of the K1 hierarchy on d1, zero guess  (Eq. TG-operator)
    5. x += P0 e
    6. nu2 relaxation sweeps on K0.

The V-cycle on level l >= 1 is the standard Galerkin cycle with R_l = P_l^T
and an exact solve on the coarsest level.  Relaxation schedules (Sec. 4):
DC-all relaxes on every level, DC-skip1 omits level 1, DC-skip0 omits
level 0.

Readings:
* Dirichlet rows are decoupled identity rows in every assembled operator, so
  the preconditioner inverts that block exactly: z = r on Dirichlet DoFs.
* The coarsest operator is singular (enclosed flow: constant pressure); its
  exact solve uses the bordered matrix [K_L n; n^T 0], n the pressure null
  vector carried down the hierarchy.
* SV pressure transfers: P0^p duplicates each continuous vertex value into
  the discontinuous DoFs at that vertex; R0^p = Mcg^-1 Pi^T M_dg is the L2
  projection applied to the pressure residual vector, with Mcg^-1 taken as a
  fixed-degree Chebyshev-Jacobi iteration on the Wathen interval.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .vanka import VankaLevel
from . import dlsc as _dlsc

DC_ALL, DC_SKIP1, DC_SKIP0 = 0, 1, 2
VANKA, DLSC, VANKA_KRYLOV = 0, 1, 2


def krylov_relax(K, x, b, precond, k):
    """Krylov-wrapped relaxation (Sec. 3.3.1): k steps of flexible GMRES on
    K e = b - K x from e = 0, right-preconditioned by `precond` (one Vanka
    sweep, undamped, per step), Arnoldi by modified Gram-Schmidt; returns
    x + Z y with y the least-squares minimiser of ||beta e1 - H y||.  The
    steps stop early at an exact (lucky) breakdown."""
    r = b - K @ x
    beta = np.linalg.norm(r)
    if beta == 0.0:
        return x
    V = [r / beta]
    Z = []
    H = np.zeros((k + 1, k))
    steps = 0
    for j in range(k):
        z = precond(V[j])
        Z.append(z)
        w = K @ z
        for i in range(j + 1):
            H[i, j] = w @ V[i]
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        steps = j + 1
        if H[j + 1, j] == 0.0:
            break
        V.append(w / H[j + 1, j])
    g = np.zeros(steps + 1)
    g[0] = beta
    y = np.linalg.lstsq(H[:steps + 1, :steps], g, rcond=None)[0]
    e = np.zeros_like(x)
    for j in range(steps):
        e = e + y[j] * Z[j]
    return x + e


class Params:
    def __init__(self, schedule=DC_ALL, nu1=1, nu2=1, eta_u=1.0, eta_p=1.0,
                 omega=None, relax=None, cheb_deg=(3, 3, 6), mcg_deg=32, dlsc_sweeps=2):
        self.schedule = schedule
        self.nu1, self.nu2 = nu1, nu2
        self.eta_u, self.eta_p = eta_u, eta_p
        self.omega = omega          # list per relaxed level (default 1.0)
        self.relax = relax          # list per relaxed level (default Vanka)
        self.cheb_deg = cheb_deg
        self.mcg_deg = mcg_deg
        self.dlsc_sweeps = dlsc_sweeps


def chebyshev_jacobi(M, b, lo, hi, degree):
    """x ~= M^-1 b by `degree` steps of the Chebyshev semi-iteration for the
    Jacobi-preconditioned system D^-1 M x = D^-1 b, eigenvalues of D^-1 M in
    [lo, hi], zero initial guess (Saad, Iterative Methods, Alg. 12.1)."""
    return _dlsc.chebyshev(lambda y: M @ y, b, lo, hi, degree, dinv=1.0 / M.diagonal())


class Oracle:
    """Holds the per-level data of one problem and applies the DC cycle."""

    def __init__(self, prob, params):
        self.prob = prob
        self.p = params
        L = prob.nlevels
        self.L = L
        self.K = [k.tocsr() for k in prob.K]
        self.Pm = [p.tocsr() for p in prob.P]
        self.R = [p.T.tocsr() for p in self.Pm]
        nrel = L - 1
        self.omega = list(params.omega) if params.omega is not None else [1.0] * nrel
        self.relax = list(params.relax) if params.relax is not None else [VANKA] * nrel
        self.vanka = {}
        self.dl = {}
        for l in range(nrel):
            if self.relax[l] in (VANKA, VANKA_KRYLOV):
                self.vanka[l] = VankaLevel(self.K[l], prob.patches[l])
            else:
                self.dl[l] = _dlsc.DLSCLevel(prob, l, params)
        # bordered coarsest matrix, LU with partial pivoting
        KL = self.K[-1].toarray()
        nL = KL.shape[0]
        n = prob.coarse_null
        Bd = np.zeros((nL + 1, nL + 1))
        Bd[:nL, :nL] = KL
        Bd[:nL, nL] = n
        Bd[nL, :nL] = n
        self.coarse_lu = sla.lu_factor(Bd)
        self.dirichlet = prob.dirichlet
        off = prob.field_off[0]
        d = prob.dim
        self.eta = np.concatenate([np.full(off[d] - off[0], params.eta_u),
                                   np.full(off[d + 1] - off[d], params.eta_p)])

    # -- pieces -------------------------------------------------------------
    def relax_level(self, l, x, b, sweeps):
        if self.relax[l] == VANKA_KRYLOV:
            # `sweeps` inner FGMRES steps, one Vanka sweep each
            return krylov_relax(self.K[l], x, b, self.vanka[l].apply, sweeps) if sweeps > 0 else x
        for _ in range(sweeps):
            if self.relax[l] == VANKA:
                x = self.vanka[l].sweep(self.K[l], x, b, self.omega[l])
            else:
                x = self.dl[l].sweep(x, b)
        return x

    def coarse_solve(self, b):
        nL = b.size
        rhs = np.concatenate([b, [0.0]])
        return sla.lu_solve(self.coarse_lu, rhs)[:nL]

    def restrict0(self, d):
        """R0 d: injection for TH; for SV velocity injection and the L2
        projection of the discontinuous pressure residual."""
        prob = self.prob
        if prob.disc == 0:
            return self.R[0] @ d
        dim = prob.dim
        off0, off1 = prob.field_off[0], prob.field_off[1]
        nv = off0[dim]
        out = np.zeros(self.K[1].shape[0])
        out[:nv] = d[:nv]
        rhs = prob.R0p @ d[off0[dim]:off0[dim + 1]]
        lo, hi = prob.mcg_bounds
        out[off1[dim]:off1[dim + 1]] = chebyshev_jacobi(prob.Mcg, rhs, lo, hi, self.p.mcg_deg)
        return out

    # -- cycles ---------------------------------------------------------------
    def vcycle(self, l, b):
        """Galerkin V(nu1, nu2) cycle on level l >= 1, zero initial guess."""
        if l == self.L - 1:
            return self.coarse_solve(b)
        skip = self.p.schedule == DC_SKIP1 and l == 1
        x = np.zeros_like(b)
        if not skip:
            x = self.relax_level(l, x, b, self.p.nu1)
        r = b - self.K[l] @ x
        e = self.vcycle(l + 1, self.R[l] @ r)
        x = x + self.Pm[l] @ e
        if not skip:
            x = self.relax_level(l, x, b, self.p.nu2)
        return x

    def apply(self, r):
        """z = M_dc^-1 r (Eq. TG-operator-full with gamma = 1)."""
        r = np.asarray(r, dtype=np.float64)
        skip0 = self.p.schedule == DC_SKIP0
        x = np.zeros_like(r)
        if not skip0:
            x = self.relax_level(0, x, r, self.p.nu1)
        if self.L == 1:
            z = x
        else:
            d = self.eta * (r - self.K[0] @ x)
            e = self.vcycle(1, self.restrict0(d))
            x = x + self.Pm[0] @ e
            if not skip0:
                x = self.relax_level(0, x, r, self.p.nu2)
            z = x
        z = z.copy()
        z[self.dirichlet] = r[self.dirichlet]
        return z
