"""The synthetic workloads and their solver parameters.

Each entry names the problem (mesh, element pair, boundary conditions,
right-hand side, seeds) and the solver parameters of the defect-correction
cycle.  Parameter sources: eta from the optimal-damping table for Taylor-Hood
(Sec. 4.1: DC-all Vanka, 2D structured 0.75, 3D 1.00) and the
(omega_0, eta_p) table for Scott-Vogelius (Sec. 4.2); the stationary Vanka
damping omega for Taylor-Hood from the brute-force search of Sec. 4
(run by the oracle's search tool on the 16^2 and 64^2 lid/manufactured
problems: 0.70 and 0.55; the larger problem's value is kept).
"""
from . import mesh as M, stokes

# cycle parameters ------------------------------------------------------------
TH2D_VANKA = dict(schedule=0, nu1=1, nu2=1, eta_u=0.75, eta_p=0.75, omega=0.55)
SV2D_VANKA = dict(schedule=0, nu1=1, nu2=1, eta_u=1.0, eta_p=2.68, omega0=0.78, omega=0.55)
SV2D_VANKA_DLSC = dict(schedule=0, nu1=1, nu2=1, eta_u=1.0, eta_p=2.96, omega0=0.87, omega=1.0)

FGMRES = dict(rtol=1e-8, restart=30, maxit=600)
# the paper's own solver setting (Sec. 4): FGMRES(20), residual reduced by 1e10
FGMRES_PAPER = dict(rtol=1e-10, restart=20, maxit=600)


def th2d_dlsc(nlevels):
    """DLSC-AMG for Taylor-Hood (Sec. 3.3.2, Sec. 4.1): DLSC relaxation on
    every level, Mu = diag(velocity mass) on K0 and I on the P1isoP2
    hierarchy, eta = 1.00 (Table p2p1_taus, DLSC, DC-all, 2D structured),
    two sweeps per relaxation call with the Table lsd_dgs_config degrees."""
    return dict(schedule=0, nu1=1, nu2=1, eta_u=1.0, eta_p=1.0, omega=1.0, relax=[1] * (nlevels - 1),
                dlsc_sweeps=2)


def c1():
    """2D Taylor-Hood 16x16, lid-driven cavity, f = 0, nu = 1."""
    return stokes.build_th(M.unit_square(16), nu=1.0, bc="lid", rhs="zero", name="C1 TH2D 16^2 lid")


def c2(n=256):
    """2D Taylor-Hood 256x256, manufactured smooth solution, ~6 levels."""
    return stokes.build_th(M.unit_square(n), nu=1.0, bc="noslip", rhs="manufactured",
                           max_levels=6, name=f"C2 TH2D {n}^2 manufactured")


def c3(n=128):
    """2D Scott-Vogelius P2/P1disc on the Alfeld split of a 128x128 mesh,
    interior vertices perturbed by U(-0.2h, 0.2h), f nodal N(0,1)."""
    return stokes.build_sv(n, nu=1.0, perturb=0.2, seed_perturb=3001, seed_f=3002, name=f"C3 SV2D {n}^2")


def sv_vanka_dlsc(nlevels):
    """Vanka on level 0, DLSC on levels >= 1 (Table p2p1disc_params)."""
    return dict(SV2D_VANKA_DLSC, relax=[0] + [1] * (nlevels - 2))


# 3D: eta = 1.00 (Sec. 4.1 table, 3D structured Vanka); omega from the
# brute-force search on the 6^3 cavity (0.70: 10 iterations; 0.55: 11)
TH3D_VANKA = dict(schedule=0, nu1=1, nu2=1, eta_u=1.0, eta_p=1.0, omega=0.70)


def c4(n=32):
    """3D Taylor-Hood P2/P1, unit cube n^3 hexes split into 6 Kuhn tetrahedra,
    lid-driven cavity (u = (1,0,0) strictly inside the top face), f = 0."""
    return stokes.build_th(M.unit_cube(n), nu=1.0, bc="lid", rhs="zero", name=f"C4 TH3D {n}^3 lid")


def c5_instances(count=64, lo=32, hi=192, seed=5000):
    """Batched workload: `count` independent 2D Taylor-Hood problems on n x n
    unit squares, n ~ U{lo..hi}, nu = 10^U(-2, 2), b_u ~ N(0,1) on free rows,
    b_p = 0, no-slip walls; instance k draws from seed + k."""
    from . import rng
    ns = rng.integers(seed, count, lo, hi)
    lognu = rng.uniform(seed + 10**6, count, -2.0, 2.0)
    return [(int(ns[k]), float(10.0 ** lognu[k]), seed + k) for k in range(count)]


def _c5_one(args):
    k, n, nu, s = args
    return stokes.build_th(M.unit_square(n), nu=nu, bc="noslip", rhs="random_b", seed=s,
                           name=f"C5[{k}] TH2D {n}^2 nu={nu:.3g}")


def c5(count=64, lo=32, hi=192, seed=5000, workers=None):
    """The batched workload; instances are built in a spawn-context process
    pool when workers > 1 (default: the host's cores)."""
    import os
    jobs = [(k, n, nu, s) for k, (n, nu, s) in enumerate(c5_instances(count, lo, hi, seed))]
    workers = workers if workers is not None else min(len(jobs), os.cpu_count() or 1)
    if workers <= 1:
        return [_c5_one(j) for j in jobs]
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    # largest first for load balance, results back in instance order
    order = sorted(range(len(jobs)), key=lambda i: -jobs[i][1])
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        built = list(ex.map(_c5_one, [jobs[i] for i in order]))
    out = [None] * len(jobs)
    for i, p in zip(order, built):
        out[i] = p
    return out


# HO-AMG (Alg. 1 applied to K0, the remark of Sec. 3.2): a standard V-cycle
# on K0, so eta = 1; omega from the oracle's search on the 16^2 and 32^2 lid
# problems (0.70 best on both).
HO_AMG_TH2D = dict(schedule=0, nu1=1, nu2=1, eta_u=1.0, eta_p=1.0, omega=0.70)


def ho_amg_th2d(n=16):
    return stokes.build_ho_amg(M.unit_square(n), nu=1.0, bc="lid", name=f"HO-AMG TH2D {n}^2 lid")


# Reduced sizes of the configs, on which the FP64 oracle's FGMRES solve
# finishes in seconds (the FP32-preconditioned solution is compared with the
# oracle's there): name -> (problem builder, parameter builder, note).
def reduced_cases():
    return {
        "C1": (c1, lambda pr: TH2D_VANKA, "full size"),
        "C2": (lambda: c2(64), lambda pr: TH2D_VANKA, "64^2 (full size 256^2)"),
        "C2 DLSC-AMG": (lambda: c2(64), lambda pr: th2d_dlsc(pr.nlevels), "64^2 (full size 256^2)"),
        "C3 Vanka": (lambda: c3(32), lambda pr: SV2D_VANKA, "32^2 (full size 128^2)"),
        "C3 Vanka + DLSC": (lambda: c3(32), lambda pr: sv_vanka_dlsc(pr.nlevels), "32^2 (full size 128^2)"),
        "C4": (lambda: c4(8), lambda pr: TH3D_VANKA, "8^3 (full size 32^3)"),
    }
