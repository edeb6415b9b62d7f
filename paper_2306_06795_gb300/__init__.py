"""Python binding of libstokes_dcamg.so (include/stokes_dcamg.h).

Argument marshalling only: every step of the solve runs in the CUDA library.
The functions carry the C names (``stokes_setup``, ``stokes_factor_patches``,
``stokes_vcycle``, ``stokes_fgmres_solve`` ...); device vectors are passed as
torch CUDA tensors (FP64, contiguous), problems as objects with the fields
of ``stokes_problem`` (see ``problems.stokes.Problem``).  Importing this
module loads the library and raises if it is missing: there is no CPU path.
"""
import ctypes as C
import os

import numpy as np

from .build import LIB, build as _build

# ---------------------------------------------------------------- constants
STOKES_OK = 0
STOKES_NOT_CONVERGED = 1
STOKES_ERR_INVALID_ARG = -1
STOKES_ERR_CUDA = -2
STOKES_ERR_OOM = -3
STOKES_ERR_SINGULAR_PATCH = -4
STOKES_ERR_NAN = -5
STOKES_ERR_STATE = -6
STOKES_TH, STOKES_SV = 0, 1
STOKES_DC_ALL, STOKES_DC_SKIP1, STOKES_DC_SKIP0 = 0, 1, 2
STOKES_RELAX_VANKA, STOKES_RELAX_DLSC, STOKES_RELAX_VANKA_KRYLOV = 0, 1, 2
STOKES_PRECOND_DC, STOKES_PRECOND_BTP = 0, 1
STOKES_FP32, STOKES_FP64 = 0, 1
STOKES_KERNEL_VANKA_APPLY, STOKES_KERNEL_SCATTER, STOKES_KERNEL_SPMV, STOKES_KERNEL_DC_RESIDUAL = range(4)
(STOKES_OP_SPMV, STOKES_OP_SPMV_F64, STOKES_OP_RESIDUAL, STOKES_OP_RESTRICT,
 STOKES_OP_PROLONG, STOKES_OP_VANKA, STOKES_OP_RELAX, STOKES_OP_COARSE) = range(8)

# Chebyshev degrees of the DLSC stages (momentum, continuity, pressure
# correction) by dimension, Table lsd_dgs_config
DLSC_DEGREES = {2: (3, 3, 6), 3: (4, 4, 16)}

EXPORTS = ["stokes_setup", "stokes_factor_patches", "stokes_vcycle", "stokes_fgmres_solve",
           "stokes_fgmres_solve_host", "stokes_level_op", "stokes_num_levels", "stokes_level_size",
           "stokes_cycle_bytes", "stokes_sweep_factor_bytes", "stokes_time_kernel",
           "stokes_kernel_launches", "stokes_vanka_noalloc", "stokes_inject_pipeline_error", "stokes_destroy",
           "stokes_autotune", "stokes_autotune_report", "stokes_galerkin", "stokes_csr_free", "stokes_sa_strength",
           "stokes_sa_tentative", "stokes_sa_smooth", "stokes_vanka_patches", "stokes_patch_lists_free",
           "stokes_status_string", "stokes_last_error"]


# ---------------------------------------------------------------- structs
class stokes_csr(C.Structure):
    _fields_ = [("nrows", C.c_int32), ("ncols", C.c_int32), ("nnz", C.c_int64),
                ("rowptr", C.POINTER(C.c_int64)), ("col", C.POINTER(C.c_int32)),
                ("val", C.POINTER(C.c_double))]


class stokes_patches(C.Structure):
    _fields_ = [("npatch", C.c_int32), ("ptr", C.POINTER(C.c_int64)), ("dof", C.POINTER(C.c_int32)),
                ("nvel", C.POINTER(C.c_int32)), ("npres", C.POINTER(C.c_int32))]


class stokes_btp(C.Structure):
    _fields_ = [("nlevels_a", C.c_int32), ("A", C.POINTER(stokes_csr)), ("PA", C.POINTER(stokes_csr)),
                ("B", C.POINTER(stokes_csr)), ("nlevels_m", C.c_int32), ("M", C.POINTER(stokes_csr)),
                ("PM", C.POINTER(stokes_csr)), ("Minv", C.POINTER(stokes_csr))]


class stokes_problem(C.Structure):
    _fields_ = [("dim", C.c_int32), ("disc", C.c_int32), ("nlevels", C.c_int32),
                ("field_off", C.POINTER(C.c_int64)), ("K", C.POINTER(stokes_csr)),
                ("P", C.POINTER(stokes_csr)), ("patches", C.POINTER(stokes_patches)),
                ("coarse_null", C.POINTER(C.c_double)), ("dirichlet", C.POINTER(C.c_uint8)),
                ("R0p", C.POINTER(stokes_csr)), ("Mcg", C.POINTER(stokes_csr)),
                ("mcg_lo", C.c_double), ("mcg_hi", C.c_double),
                ("lambda_A", C.POINTER(C.c_double)), ("lambda_S", C.POINTER(C.c_double)),
                ("btp", C.POINTER(stokes_btp)), ("Mu_diag", C.POINTER(C.c_double))]


class stokes_params(C.Structure):
    _fields_ = [("schedule", C.c_int32), ("nu1", C.c_int32), ("nu2", C.c_int32),
                ("eta_u", C.c_double), ("eta_p", C.c_double), ("omega", C.POINTER(C.c_double)),
                ("relax", C.POINTER(C.c_int32)), ("cheb_deg", C.c_int32 * 3), ("dlsc_sweeps", C.c_int32),
                ("mcg_deg", C.c_int32), ("precision", C.c_int32), ("preconditioner", C.c_int32),
                ("btp_steps", C.c_int32), ("factor_tcgen05", C.c_int32)]


class stokes_solve_info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("status", C.c_int32), ("true_relres", C.c_double)]


# ---------------------------------------------------------------- loading
def _load():
    if not os.path.exists(LIB):
        raise ImportError(f"libstokes_dcamg.so is not built ({LIB}); run __graft_entry__.build()")
    lib = C.CDLL(LIB)
    vp = C.c_void_p
    lib.stokes_setup.argtypes = [C.POINTER(C.POINTER(stokes_problem)), C.c_int32, C.POINTER(stokes_params), vp,
                                 C.POINTER(vp)]
    lib.stokes_factor_patches.argtypes = [vp, C.POINTER(C.c_int64)]
    lib.stokes_vcycle.argtypes = [vp, vp, vp]
    lib.stokes_fgmres_solve.argtypes = [vp, vp, vp, C.c_double, C.c_int32, C.c_int32, C.POINTER(stokes_solve_info)]
    lib.stokes_fgmres_solve_host.argtypes = [vp, vp, vp, C.c_double, C.c_int32, C.c_int32,
                                             C.POINTER(stokes_solve_info)]
    lib.stokes_level_op.argtypes = [vp, C.c_int32, C.c_int32, vp, vp, vp]
    lib.stokes_num_levels.argtypes = [vp]
    lib.stokes_level_size.argtypes = [vp, C.c_int32]
    lib.stokes_level_size.restype = C.c_int64
    lib.stokes_cycle_bytes.argtypes = [vp]
    lib.stokes_cycle_bytes.restype = C.c_double
    lib.stokes_sweep_factor_bytes.argtypes = [vp, C.c_int32]
    lib.stokes_sweep_factor_bytes.restype = C.c_double
    lib.stokes_time_kernel.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_double),
                                       C.POINTER(C.c_double)]
    lib.stokes_kernel_launches.argtypes = [vp]
    lib.stokes_kernel_launches.restype = C.c_int64
    lib.stokes_vanka_noalloc.argtypes = [vp, C.c_int32, vp, vp]
    lib.stokes_inject_pipeline_error.argtypes = [vp, C.c_int32]
    lib.stokes_destroy.argtypes = [vp]
    lib.stokes_galerkin.argtypes = [C.POINTER(stokes_csr), C.POINTER(stokes_csr), vp, C.POINTER(stokes_csr)]
    lib.stokes_galerkin.restype = C.c_int
    lib.stokes_csr_free.argtypes = [C.POINTER(stokes_csr)]
    lib.stokes_sa_strength.argtypes = [C.POINTER(stokes_csr), C.c_double, vp, C.POINTER(stokes_csr)]
    lib.stokes_sa_strength.restype = C.c_int
    lib.stokes_sa_tentative.argtypes = [C.c_int32, C.POINTER(C.c_int32), C.c_int32, C.POINTER(C.c_double), vp,
                                        C.POINTER(stokes_csr), C.POINTER(C.c_double)]
    lib.stokes_sa_tentative.restype = C.c_int
    lib.stokes_sa_smooth.argtypes = [C.POINTER(stokes_csr), C.POINTER(stokes_csr), C.c_double, vp,
                                     C.POINTER(stokes_csr)]
    lib.stokes_sa_smooth.restype = C.c_int
    lib.stokes_vanka_patches.argtypes = [C.POINTER(stokes_csr), C.POINTER(C.c_int64), C.c_int32, C.c_double, vp,
                                         C.POINTER(stokes_patches)]
    lib.stokes_vanka_patches.restype = C.c_int
    lib.stokes_patch_lists_free.argtypes = [C.POINTER(stokes_patches)]
    lib.stokes_autotune.argtypes = [vp, C.c_int32]
    lib.stokes_autotune.restype = C.c_int
    lib.stokes_autotune_report.argtypes = [vp]
    lib.stokes_autotune_report.restype = C.c_char_p
    lib.stokes_destroy.restype = None
    lib.stokes_status_string.argtypes = [C.c_int]
    lib.stokes_status_string.restype = C.c_char_p
    lib.stokes_last_error.argtypes = []
    lib.stokes_last_error.restype = C.c_char_p
    return lib


lib = _load()


class StokesError(RuntimeError):
    def __init__(self, code, where):
        msg = lib.stokes_last_error().decode()
        super().__init__(f"{where}: {lib.stokes_status_string(code).decode()} ({code}): {msg}")
        self.code = code


def _check(code, where, allow_not_converged=False):
    if code < 0 or (code > 0 and not allow_not_converged):
        raise StokesError(code, where)
    return code


# ---------------------------------------------------------------- marshalling
def _p(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


class _Keep:
    """Holds numpy arrays alive while the C structs point at them."""

    def __init__(self):
        self.refs = []

    def arr(self, a, dtype):
        a = np.ascontiguousarray(a, dtype=dtype)
        self.refs.append(a)
        return a


def _csr(keep, m):
    m = m.tocsr()
    m.sort_indices()
    rp = keep.arr(m.indptr, np.int64)
    ci = keep.arr(m.indices, np.int32)
    v = keep.arr(m.data, np.float64)
    return stokes_csr(m.shape[0], m.shape[1], m.nnz, _p(rp, C.c_int64), _p(ci, C.c_int32), _p(v, C.c_double))


def _problem(keep, pr):
    L = len(pr.K)
    Ks = (stokes_csr * L)(*[_csr(keep, k) for k in pr.K])
    Ps = (stokes_csr * (L - 1))(*[_csr(keep, p) for p in pr.P[: L - 1]])
    pas = []
    for pa in pr.patches[: L - 1]:
        ptr = keep.arr(pa.ptr, np.int64)
        dof = keep.arr(pa.dof, np.int32)
        nv = keep.arr(np.asarray(pa.nvel).reshape(-1), np.int32)
        npr = keep.arr(pa.npres, np.int32)
        pas.append(stokes_patches(pa.ptr.size - 1, _p(ptr, C.c_int64), _p(dof, C.c_int32), _p(nv, C.c_int32),
                                  _p(npr, C.c_int32)))
    Pa = (stokes_patches * (L - 1))(*pas)
    keep.refs += [Ks, Ps, Pa]
    fo = keep.arr(np.concatenate([np.asarray(o, dtype=np.int64) for o in pr.field_off]), np.int64)
    cn = keep.arr(pr.coarse_null, np.float64)
    dr = keep.arr(pr.dirichlet.astype(np.uint8), np.uint8)
    p = stokes_problem()
    p.dim, p.disc, p.nlevels = pr.dim, pr.disc, L
    p.field_off = _p(fo, C.c_int64)
    p.K = C.cast(Ks, C.POINTER(stokes_csr))
    p.P = C.cast(Ps, C.POINTER(stokes_csr))
    p.patches = C.cast(Pa, C.POINTER(stokes_patches))
    p.coarse_null = _p(cn, C.c_double)
    p.dirichlet = _p(dr, C.c_uint8)
    if getattr(pr, "R0p", None) is not None:
        r0 = _csr(keep, pr.R0p)
        mc = _csr(keep, pr.Mcg)
        keep.refs += [r0, mc]
        p.R0p = C.pointer(r0)
        p.Mcg = C.pointer(mc)
        p.mcg_lo, p.mcg_hi = pr.mcg_bounds
    if getattr(pr, "lambda_A", None) is not None:
        la = keep.arr(pr.lambda_A, np.float64)
        ls = keep.arr(pr.lambda_S, np.float64)
        p.lambda_A = _p(la, C.c_double)
        p.lambda_S = _p(ls, C.c_double)
    if getattr(pr, "Mu_diag", None) is not None:
        md = keep.arr(pr.Mu_diag, np.float64)
        p.Mu_diag = _p(md, C.c_double)
    bt = getattr(pr, "btp", None)
    if bt is not None:
        q = stokes_btp()
        As = (stokes_csr * len(bt.A))(*[_csr(keep, a) for a in bt.A])
        PAs = (stokes_csr * max(len(bt.PA), 1))(*[_csr(keep, a) for a in bt.PA])
        Bc = _csr(keep, bt.B)
        keep.refs += [As, PAs, Bc, q]
        q.nlevels_a = len(bt.A)
        q.A = C.cast(As, C.POINTER(stokes_csr))
        q.PA = C.cast(PAs, C.POINTER(stokes_csr))
        q.B = C.pointer(Bc)
        if bt.Minv is not None:
            mi = _csr(keep, bt.Minv)
            keep.refs.append(mi)
            q.Minv = C.pointer(mi)
            q.nlevels_m = 0
        else:
            Ms = (stokes_csr * len(bt.M))(*[_csr(keep, a) for a in bt.M])
            PMs = (stokes_csr * max(len(bt.PM), 1))(*[_csr(keep, a) for a in bt.PM])
            keep.refs += [Ms, PMs]
            q.nlevels_m = len(bt.M)
            q.M = C.cast(Ms, C.POINTER(stokes_csr))
            q.PM = C.cast(PMs, C.POINTER(stokes_csr))
        p.btp = C.pointer(q)
    return p


def _params(keep, prm, nlevels, dim=2):
    """prm: dict with schedule, nu1, nu2, eta_u, eta_p, omega (scalar or per
    level; omega0 overrides level 0), relax (list or None), cheb_deg (default:
    the DLSC degrees of the paper's table for the dimension, (3, 3, 6) in 2D
    and (4, 4, 16) in 3D), dlsc_sweeps, mcg_deg, precision, preconditioner,
    btp_steps, factor_tcgen05."""
    s = stokes_params()
    s.schedule = int(prm.get("schedule", 0))
    s.nu1 = int(prm.get("nu1", 1))
    s.nu2 = int(prm.get("nu2", 1))
    s.eta_u = float(prm.get("eta_u", 1.0))
    s.eta_p = float(prm.get("eta_p", 1.0))
    om = prm.get("omega", 1.0)
    om = np.full(max(nlevels - 1, 1), float(om)) if np.isscalar(om) else np.asarray(om, dtype=np.float64)
    if "omega0" in prm:
        om = om.copy()
        om[0] = prm["omega0"]
    om = keep.arr(om, np.float64)
    s.omega = _p(om, C.c_double)
    if prm.get("relax") is not None:
        rl = keep.arr(prm["relax"], np.int32)
        s.relax = _p(rl, C.c_int32)
    cd = prm.get("cheb_deg", DLSC_DEGREES[dim])
    s.cheb_deg[0], s.cheb_deg[1], s.cheb_deg[2] = (int(v) for v in cd)
    s.dlsc_sweeps = int(prm.get("dlsc_sweeps", 2))
    s.mcg_deg = int(prm.get("mcg_deg", 32))
    s.precision = int(prm.get("precision", STOKES_FP32))
    s.preconditioner = int(prm.get("preconditioner", STOKES_PRECOND_DC))
    s.btp_steps = int(prm.get("btp_steps", 2))
    s.factor_tcgen05 = int(prm.get("factor_tcgen05", 0))
    return s


# ---------------------------------------------------------------- API
def _dptr(t, n=None, what="vector"):
    """Device address of a contiguous FP64 CUDA tensor of n entries (n=None:
    any size).  Raises instead of passing the library a pointer it would read
    or write out of bounds."""
    if t is None:
        return None
    if not getattr(t, "is_cuda", False):
        raise TypeError(f"{what}: a CUDA tensor is expected")
    import torch
    if t.dtype != torch.float64:
        raise TypeError(f"{what}: FP64 expected, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what}: a contiguous tensor is expected")
    if n is not None and t.numel() != n:
        raise ValueError(f"{what}: {n} entries expected, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


class Handle:
    """Owns a stokes_handle; closed by ``stokes_destroy`` or garbage collection."""

    def __init__(self, ptr, ninst):
        self.ptr = ptr
        self.ninst = ninst

    def __del__(self):
        if getattr(self, "ptr", None):
            stokes_destroy(self)


def stokes_setup(problems, params, stream=None):
    """Build a handle for one problem or a list of problems (batched)."""
    if not isinstance(problems, (list, tuple)):
        problems = [problems]
    keep = _Keep()
    cps = [_problem(keep, pr) for pr in problems]
    arr = (C.POINTER(stokes_problem) * len(cps))(*[C.pointer(p) for p in cps])
    nl = max(len(pr.K) for pr in problems)
    prm = _params(keep, params, nl, problems[0].dim)
    out = C.c_void_p()
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    _check(lib.stokes_setup(arr, len(cps), C.byref(prm), C.c_void_p(stream), C.byref(out)), "stokes_setup")
    return Handle(out, len(cps))


def stokes_factor_patches(h):
    ns = C.c_int64(0)
    _check(lib.stokes_factor_patches(h.ptr, C.byref(ns)), "stokes_factor_patches")
    return ns.value


def stokes_vcycle(h, r, z):
    n = stokes_level_size(h, 0)
    _check(lib.stokes_vcycle(h.ptr, _dptr(r, n, "r"), _dptr(z, n, "z")), "stokes_vcycle")


def stokes_fgmres_solve(h, b, x, rtol=1e-8, restart=30, maxit=1000):
    info = (stokes_solve_info * h.ninst)()
    n = stokes_level_size(h, 0)
    rc = _check(lib.stokes_fgmres_solve(h.ptr, _dptr(b, n, "b"), _dptr(x, n, "x"), rtol, restart, maxit, info),
                "stokes_fgmres_solve", allow_not_converged=True)
    return rc, [(i.iters, i.status, i.true_relres) for i in info]


def stokes_fgmres_solve_host(h, b, x, rtol=1e-8, restart=30, maxit=1000):
    """b, x: numpy FP64 arrays in host memory (x: initial guess in, solution out)."""
    n = stokes_level_size(h, 0)
    for nm, a in (("b", b), ("x", x)):
        if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags.c_contiguous or a.size != n:
            raise ValueError(f"{nm}: a contiguous FP64 numpy array of {n} entries is expected")
    info = (stokes_solve_info * h.ninst)()
    rc = _check(lib.stokes_fgmres_solve_host(h.ptr, C.c_void_p(b.ctypes.data), C.c_void_p(x.ctypes.data), rtol,
                                             restart, maxit, info),
                "stokes_fgmres_solve_host", allow_not_converged=True)
    return rc, [(i.iters, i.status, i.true_relres) for i in info]


def _csr_out(out):
    """Copy a library-allocated CSR into a scipy CSR and release it."""
    import scipy.sparse as sp
    try:
        n, nnz = out.nrows, out.nnz
        rp = np.ctypeslib.as_array(out.rowptr, shape=(n + 1,)).copy()
        ci = np.ctypeslib.as_array(out.col, shape=(nnz,)).copy() if nnz else np.zeros(0, np.int32)
        va = np.ctypeslib.as_array(out.val, shape=(nnz,)).copy() if nnz else np.zeros(0)
    finally:
        lib.stokes_csr_free(C.byref(out))
    return sp.csr_matrix((va, ci, rp), shape=(out.nrows, out.ncols))


def _stream(stream):
    return C.c_void_p(stream) if stream else None


def stokes_galerkin(K, P, stream=None):
    """P^T K P on the device (FP64); K, P: scipy sparse matrices; returns a scipy CSR."""
    keep = _Keep()
    k = _csr(keep, K)
    p = _csr(keep, P)
    out = stokes_csr()
    _check(lib.stokes_galerkin(C.byref(k), C.byref(p), _stream(stream), C.byref(out)), "stokes_galerkin")
    return _csr_out(out)


def stokes_sa_strength(A, theta=0.0, stream=None):
    """Strength-of-connection pattern of A on the device (scipy CSR, values 1)."""
    keep = _Keep()
    a = _csr(keep, A)
    out = stokes_csr()
    _check(lib.stokes_sa_strength(C.byref(a), float(theta), _stream(stream), C.byref(out)), "stokes_sa_strength")
    return _csr_out(out)


def stokes_sa_tentative(agg, naggregates, B, stream=None):
    """Tentative prolongator of the aggregates agg (-1: none) with near-null
    vector B on the device; returns (T as scipy CSR, aggregate norms Bc)."""
    agg = np.ascontiguousarray(agg, dtype=np.int32)
    B = np.ascontiguousarray(B, dtype=np.float64)
    Bc = np.zeros(max(int(naggregates), 1))
    out = stokes_csr()
    _check(lib.stokes_sa_tentative(agg.size, agg.ctypes.data_as(C.POINTER(C.c_int32)), int(naggregates),
                                   B.ctypes.data_as(C.POINTER(C.c_double)), _stream(stream), C.byref(out),
                                   Bc.ctypes.data_as(C.POINTER(C.c_double))), "stokes_sa_tentative")
    return _csr_out(out), Bc[: int(naggregates)]


def stokes_sa_smooth(A, T, omega, stream=None):
    """Jacobi-smoothed prolongator T - omega D^-1 A T on the device (scipy CSR)."""
    keep = _Keep()
    a = _csr(keep, A)
    t = _csr(keep, T)
    out = stokes_csr()
    _check(lib.stokes_sa_smooth(C.byref(a), C.byref(t), float(omega), _stream(stream), C.byref(out)),
           "stokes_sa_smooth")
    return _csr_out(out)


def stokes_vanka_patches(K, field_off, dim, rel_tol=1e-14, stream=None):
    """Vanka patch lists of a Galerkin level on the device; returns
    (ptr int64, dof int32, nvel int32 (npatch, dim), npres int32)."""
    keep = _Keep()
    k = _csr(keep, K)
    off = np.ascontiguousarray(field_off, dtype=np.int64)
    out = stokes_patches()
    _check(lib.stokes_vanka_patches(C.byref(k), off.ctypes.data_as(C.POINTER(C.c_int64)), int(dim), float(rel_tol),
                                    _stream(stream), C.byref(out)), "stokes_vanka_patches")
    try:
        npatch = out.npatch
        ptr = np.ctypeslib.as_array(out.ptr, shape=(npatch + 1,)).copy()
        nd = int(ptr[-1])
        dof = np.ctypeslib.as_array(out.dof, shape=(nd,)).copy() if nd else np.zeros(0, np.int32)
        nvel = (np.ctypeslib.as_array(out.nvel, shape=(npatch * dim,)).copy().reshape(npatch, dim) if npatch
                else np.zeros((0, dim), np.int32))
        npres = np.ctypeslib.as_array(out.npres, shape=(npatch,)).copy() if npatch else np.zeros(0, np.int32)
    finally:
        lib.stokes_patch_lists_free(C.byref(out))
    return ptr, dof, nvel, npres


def stokes_autotune(h, reps=5):
    _check(lib.stokes_autotune(h.ptr, reps), "stokes_autotune")


def stokes_autotune_report(h):
    return lib.stokes_autotune_report(h.ptr).decode()


def stokes_level_op(h, op, level, x, b, y):
    L = stokes_num_levels(h)
    if not 0 <= level < L:
        raise ValueError(f"level {level} outside 0..{L - 1}")
    n = stokes_level_size(h, level)
    nx = ny = n
    if op in (STOKES_OP_RESTRICT, STOKES_OP_PROLONG):
        if level + 1 >= L:
            raise ValueError("no coarser level")
        nc = stokes_level_size(h, level + 1)
        nx, ny = (n, nc) if op == STOKES_OP_RESTRICT else (nc, n)
    _check(lib.stokes_level_op(h.ptr, op, level, _dptr(x, nx, "x"), _dptr(b, n, "b"), _dptr(y, ny, "y")),
           "stokes_level_op")


def stokes_num_levels(h):
    return lib.stokes_num_levels(h.ptr)


def stokes_level_size(h, level):
    return lib.stokes_level_size(h.ptr, level)


def stokes_cycle_bytes(h):
    return lib.stokes_cycle_bytes(h.ptr)


def stokes_sweep_factor_bytes(h, level):
    return lib.stokes_sweep_factor_bytes(h.ptr, level)


def stokes_time_kernel(h, which, level, reps=10):
    """Mean duration (ms) of one hot kernel launched alone after an L2
    flush, and its algorithmic bytes per launch."""
    ms = C.c_double(0)
    by = C.c_double(0)
    _check(lib.stokes_time_kernel(h.ptr, which, level, reps, C.byref(ms), C.byref(by)), "stokes_time_kernel")
    return ms.value, by.value


def stokes_kernel_launches(h):
    return lib.stokes_kernel_launches(h.ptr)


def stokes_vanka_noalloc(h, level, x, y):
    """y = M_level^-1 x with the library's fixed scratch (no device
    allocation during the call); see include/stokes_dcamg.h."""
    L = stokes_num_levels(h)
    if not 0 <= level < L:
        raise ValueError(f"level {level} outside 0..{L - 1}")
    n = stokes_level_size(h, level)
    _check(lib.stokes_vanka_noalloc(h.ptr, level, _dptr(x, n, "x"), _dptr(y, n, "y")), "stokes_vanka_noalloc")


def stokes_inject_pipeline_error(h, level):
    """Set level's bulk-copy error flag as a timed-out wait would (test
    support; every later checked call on the handle fails)."""
    _check(lib.stokes_inject_pipeline_error(h.ptr, level), "stokes_inject_pipeline_error")


def stokes_destroy(h):
    if h.ptr:
        lib.stokes_destroy(h.ptr)
        h.ptr = None


def build():
    """Compile libstokes_dcamg.so for sm_103a (in-tree)."""
    return _build()
