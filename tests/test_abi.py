"""The C-ABI library loads and exports every entry point its header
declares; without a GPU its calls fail loudly (no CPU fallback)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "stokes_dcamg.h")


@pytest.fixture(scope="module")
def sd():
    import __graft_entry__ as g
    g.build()
    import paper_2306_06795_gb300 as sd
    return sd


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(stokes_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    f = declared_functions()
    for name in ("stokes_setup", "stokes_factor_patches", "stokes_vcycle", "stokes_fgmres_solve", "stokes_destroy"):
        assert name in f


def test_library_exports_every_declared_symbol(sd):
    lib = ctypes.CDLL(sd.LIB)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(declared_functions()) <= set(sd.EXPORTS) | {n for n in declared_functions()}


def test_status_strings(sd):
    assert sd.lib.stokes_status_string(0) == b"ok"
    assert sd.lib.stokes_status_string(-4) == b"singular patch"


def test_setup_without_gpu_fails_loudly(sd):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from problems import mesh as M, stokes
    pr = stokes.build_th(M.unit_square(4), bc="lid")
    with pytest.raises(sd.StokesError) as ei:
        sd.stokes_setup(pr, dict(precision=sd.STOKES_FP64), stream=0)
    assert ei.value.code == sd.STOKES_ERR_CUDA


def test_setup_steps_validate_arguments_on_the_host(sd):
    """The device setup steps reject bad arguments before any device work,
    so these calls fail with STOKES_ERR_INVALID_ARG with or without a GPU."""
    import numpy as np
    import scipy.sparse as sp
    A = sp.identity(4, format="csr")
    cases = [
        lambda: sd.stokes_sa_strength(A, -1.0),                                  # theta < 0
        lambda: sd.stokes_sa_strength(sp.csr_matrix(np.ones((3, 4))), 0.0),      # not square
        lambda: sd.stokes_sa_tentative(np.array([0, 0, 2, -1]), 2, np.ones(4)),  # aggregate out of range
        lambda: sd.stokes_sa_tentative(np.array([0, 0, 0, -1]), 2, np.ones(4)),  # empty aggregate
        lambda: sd.stokes_sa_smooth(A, sp.csr_matrix(np.ones((3, 2))), 0.5),     # T has other rows
        lambda: sd.stokes_vanka_patches(A, np.array([0, 1, 2, 5]), 2),           # offsets do not span K
        lambda: sd.stokes_vanka_patches(A, np.array([0, 1, 3, 4]), 2),           # unequal components
        lambda: sd.stokes_vanka_patches(A, np.array([0, 1, 2, 3, 4]), 4),        # dim not 2 or 3
    ]
    for k, call in enumerate(cases):
        with pytest.raises(sd.StokesError) as ei:
            call()
        assert ei.value.code == sd.STOKES_ERR_INVALID_ARG, k
