"""The device route of the setup step (Alg. 1, Sec. 3.2; patch lists of
Sec. 3.3.1): the same hierarchy as stokes.HostSteps, with the strength of
connection, the tentative and the smoothed prolongators, the Galerkin
products and the Galerkin-level Vanka patch lists computed by the
library's device setup steps (stokes_sa_strength, stokes_sa_tentative,
stokes_sa_smooth, stokes_galerkin, stokes_vanka_patches).  The greedy
aggregation (sequential in natural order: a parallel aggregation would
build a different hierarchy) and the Lanczos estimate of rho(D^-1 A) behind
the smoothing weight stay on the host.  The binding module is passed in, so
this package never imports the CUDA library itself.

    steps = DeviceSteps(paper_2306_06795_gb300)
    problem = stokes.build_th(mesh, ..., steps=steps)
"""
import numpy as np

from . import sa, stokes


class DeviceSteps:
    def __init__(self, sd, stream=None):
        self.sd = sd
        self.stream = stream

    def sa_field(self, A, B, max_levels, max_coarse=50, theta=0.0):
        """sa.sa_field with the strength, tentative prolongator, smoothing and
        Galerkin product on the device."""
        sd = self.sd
        As, Ps, Bs = [A.tocsr()], [], [B]
        while len(As) < max_levels and As[-1].shape[0] > max_coarse:
            Ak = As[-1]
            excl = sa.isolated_rows(Ak)
            S = sd.stokes_sa_strength(Ak, theta, stream=self.stream)
            agg, na = sa.aggregate(S, excl)
            if na == 0 or na >= Ak.shape[0]:
                break
            T, Bc = sd.stokes_sa_tentative(agg, na, Bs[-1], stream=self.stream)
            omega = (4.0 / 3.0) / sa.rho_DinvA(Ak, ~excl)
            P = sd.stokes_sa_smooth(Ak, T, omega, stream=self.stream)
            Ac = sd.stokes_galerkin(Ak, P, stream=self.stream)
            Ps.append(P)
            As.append(Ac)
            Bs.append(Bc)
        return Ps, As, Bs

    def galerkin(self, K, P):
        return self.sd.stokes_galerkin(K, P, stream=self.stream)

    def patches(self, K, off, d):
        ptr, dof, nvel, npres = self.sd.stokes_vanka_patches(K, off, d, stream=self.stream)
        return stokes.Patches(ptr.astype(np.int64), dof.astype(np.int32), nvel.astype(np.int32),
                              npres.astype(np.int32))
