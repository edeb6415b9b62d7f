"""Device-side Galerkin product of the AMG setup (Alg. 1, K_{l+1} =
P_l^T K_l P_l) against the host product of the same factors, on the 2D
P1isoP2 and 3D hierarchies, and bitwise repeatability."""
import numpy as np
import pytest

from problems import configs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sd():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2306_06795_gb300 as sd
    return sd


@pytest.mark.parametrize("make", [lambda: configs.c2(32), lambda: configs.c4(6)])
def test_galerkin_matches_host_product(sd, make):
    pr = make()
    for l in range(1, pr.nlevels - 1):
        K, P = pr.K[l].tocsr(), pr.P[l].tocsr()
        C = sd.stokes_galerkin(K, P)
        ref = (P.T @ K @ P).tocsr()
        D = (C - ref).tocsr()
        scale = np.abs(ref.data).max()
        assert D.nnz == 0 or np.abs(D.data).max() <= 1e-13 * scale
        # sorted, unique columns per row
        for i in range(0, C.shape[0], max(1, C.shape[0] // 50)):
            cols = C.indices[C.indptr[i]:C.indptr[i + 1]]
            assert np.all(np.diff(cols) > 0)
        C2 = sd.stokes_galerkin(K, P)
        assert np.array_equal(C.indptr, C2.indptr) and np.array_equal(C.indices, C2.indices)
        assert np.array_equal(C.data, C2.data)
