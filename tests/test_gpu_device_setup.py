"""The device route of the setup step (Alg. 1 with the library's device
strength, tentative and smoothed prolongators, Galerkin products and
Galerkin-level patch lists; problems/device_setup.py) against the host
route: the same hierarchy (patterns and patch lists equal, values to the
last bits of a fixed but different summation order), and the FP64 cycle on
the device-built hierarchy equal to the oracle's cycle on that same
hierarchy to 1e-12; the FP32-preconditioned solve takes the host route's
iteration count."""
import numpy as np
import pytest

from problems import configs, device_setup, mesh as M, stokes
from tests.helpers import make_oracle, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sd():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2306_06795_gb300 as sd
    return sd


def _same_csr(A, B, tol):
    A, B = A.tocsr(), B.tocsr()
    A.sort_indices()
    B.sort_indices()
    assert A.shape == B.shape
    assert np.array_equal(A.indptr, B.indptr) and np.array_equal(A.indices, B.indices)
    assert np.max(np.abs(A.data - B.data)) <= tol * np.max(np.abs(B.data))


@pytest.mark.parametrize("case", ["c1", "th2d_32", "th3d_4"])
def test_device_route_builds_the_hierarchy_and_the_cycle_matches_the_oracle(sd, case):
    mk = {"c1": lambda steps: stokes.build_th(M.unit_square(16), bc="lid", steps=steps),
          "th2d_32": lambda steps: stokes.build_th(M.unit_square(32), bc="noslip", rhs="manufactured", steps=steps),
          "th3d_4": lambda steps: stokes.build_th(M.unit_cube(4), bc="lid", steps=steps)}[case]
    prm = dict(configs.TH2D_VANKA if case != "th3d_4" else configs.TH3D_VANKA)
    host = mk(stokes.HostSteps)
    dev = mk(device_setup.DeviceSteps(sd))
    assert dev.nlevels == host.nlevels
    for l in range(host.nlevels):
        _same_csr(dev.K[l], host.K[l], 1e-12)
    for l in range(host.nlevels - 1):
        _same_csr(dev.P[l], host.P[l], 1e-12)
        for f in ("ptr", "dof", "nvel", "npres"):
            assert np.array_equal(np.asarray(getattr(dev.patches[l], f)), np.asarray(getattr(host.patches[l], f)))
    h = sd.stokes_setup(dev, dict(prm, precision=sd.STOKES_FP64))
    sd.stokes_factor_patches(h)
    r = np.random.default_rng(61).standard_normal(dev.b.size)
    z = torch.empty(r.size, dtype=torch.float64, device="cuda")
    sd.stokes_vcycle(h, torch.tensor(r, device="cuda"), z)
    torch.cuda.synchronize()
    assert rel(z.cpu().numpy(), make_oracle(dev, prm).apply(r)) < 1e-12
    its = []
    for pr in (host, dev):
        h32 = sd.stokes_setup(pr, dict(prm, precision=sd.STOKES_FP32))
        sd.stokes_factor_patches(h32)
        b = torch.tensor(pr.b, dtype=torch.float64, device="cuda")
        x = torch.zeros_like(b)
        rc, info = sd.stokes_fgmres_solve(h32, b, x, rtol=1e-8, restart=30, maxit=300)
        assert rc == sd.STOKES_OK and info[0][2] <= 1e-8
        its.append(info[0][0])
    assert its[0] == its[1]
