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
