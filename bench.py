"""Benchmark of the GB300 solve phase: FP32-preconditioned defect-correction
AMG + FP64 FGMRES on the 2D Taylor-Hood P2/P1 256x256 manufactured-solution
problem (592,387 DoFs, 6 levels).

One step = one full solve of K0 x = b to a 1e-8 relative true residual from
x0 = 0: batched Vanka factorisation of every level (stokes_factor_patches)
followed by stokes_fgmres_solve (FGMRES(30), every iteration one captured
DC-cycle graph + FP64 SpMV + CGS2 orthogonalisation).  Inputs stay resident
in HBM; the cycle's working set (~1 GB) is far above L2, so no flush is
needed between steps.

Lines: the default arm prints the GPU line (value = solves/s over all ranks;
N > 1 runs N independent replicas, scaling "weak").  At N = 1 the line also
carries, untimed by the headline: the FP64-preconditioned form, the
Krylov-wrapped and BTP variants, the paper's own solver setting on C2
(FGMRES(20), residual reduced by 1e10), compact records of the other configs
(C1, C2 with DLSC-AMG, C3 with Vanka and with Vanka + DLSC and the
divergence of its solution, C4 with stationary and Krylov-wrapped Vanka, the
C5 batch), the FP32-preconditioned solution's error against the oracle's
solution on reduced sizes, and the CPU baseline (the oracle on the host
cores, single thread and all cores).  --impl reference times the FP64 CPU
oracle on a bounded sample on rank 0 only.
"""
import os

# the CPU oracle runs single-threaded so that its core count is exact
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = ("2D Taylor-Hood P2/P1 Stokes, unit square 256x256 squares split by the (x,y)-(x+h,y+h) diagonal, "
            "manufactured u = curl(sin^2(pi x) sin^2(pi y)), p = cos(pi x) cos(pi y); FP32 DC-all V(1,1) "
            "additive-Vanka cycle on the P1isoP2/P1 SA hierarchy, FGMRES(30) to 1e-8 true relative residual")
METRIC = "Stokes solves/s to 1e-8 rel-res (FP32 DC-AMG preconditioned FGMRES)"
# dram__bytes_read.sum + dram__bytes_write.sum of one level-0 FP32 apply launch from an ncu capture,
# keyed by the SHA-256 of the kernel's sources at capture time: when the sources differ the figure
# no longer describes the kernel and the bench line reports traffic as null
APPLY_L0_TRAFFIC = {"dram_bytes": 84884736 + 2289152, "sources": ["vanka.cu", "tma.cuh", "common.cuh"],
                    "sha256": "09bf6c6f8d441c37d0f673d37e6aa8844387fabcfc082ab9707e294f42b20512"}


def apply_traffic():
    """The recorded DRAM bytes of the roofline kernel if its sources are
    unchanged since the capture, else None."""
    import hashlib
    hsh = hashlib.sha256()
    for f in APPLY_L0_TRAFFIC["sources"]:
        with open(os.path.join(ROOT, "paper_2306_06795_gb300", "csrc", f), "rb") as fh:
            hsh.update(fh.read())
    return APPLY_L0_TRAFFIC["dram_bytes"] if hsh.hexdigest() == APPLY_L0_TRAFFIC["sha256"] else None


def fgmres_leg(n, nnz_k0, iters, restart, outside_ms, peak_gbs):
    """The FGMRES leg outside the cycle, per iteration: algorithmic bytes and
    FP64 FMAs of the Arnoldi step j (NK = j + 1 basis vectors): the FP64 K0
    SpMV (values, columns, row pointers, z gathered, w written), the three
    fused Gram-Schmidt passes (dots: NK columns + w; axpy + dots: NK columns +
    w read and written; axpy + norm: the same) and the next Krylov vector (w
    read, v written in FP64 and FP32); 4 NK + 1 FMAs per row plus one per
    nonzero of K0.  Against the measured time outside the cycle."""
    steps = [(j % restart) + 1 for j in range(iters)]
    byt = sum(nnz_k0 * 12 + 4 * (n + 1) + 16 * n + (3 * nk + 5) * 8 * n + 20 * n for nk in steps) / iters
    dfma = sum(nnz_k0 + (4 * nk + 1) * n for nk in steps) / iters
    return {"outside_cycle_ms_per_iter": outside_ms, "bytes_per_iter": byt, "dfma_per_iter": dfma,
            "GBps": byt / outside_ms / 1e6, "frac_of_measured_hbm": byt / outside_ms / 1e6 / peak_gbs,
            "T_dfma_per_s": dfma / outside_ms / 1e9,
            "note": "time outside the cycle = (step - factorisation - iterations x cycle) / iterations; "
                    "includes the restart's residual and x += Z y"}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"stokes_bench_clocks_{os.getpid()}.csv")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        self.skip = 0
        if self.proc is not None:
            # wait (at most 5 s) until sampling runs, then count only the
            # samples taken from here on, i.e. inside the timed region
            t0 = time.time()
            while time.time() - t0 < 5.0 and self._lines() == 0 and self.proc.poll() is None:
                time.sleep(0.02)
            self.skip = self._lines()

    def _lines(self):
        try:
            self.f.flush()
            with open(self.path) as g:
                return sum(1 for _ in g)
        except Exception:
            return 0

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for k_line, line in enumerate(open(self.path)):
            if k_line < self.skip:
                continue
            p = [x.strip() for x in line.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                smax.append(float(p[1]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if p[4 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------- CPU oracle
# The oracle runs in spawned worker processes, one thread each (the
# environment above pins the BLAS threads), only in the cpu_baseline leg and
# in the reference arm.
_C2_PROBLEM = []  # the C2 problem, built once per worker process (host setup, not timed)


def _oracle_c2_sample(with_cycle=True):
    """Bounded sample of the C2 solve by the FP64 oracle: its setup (dense
    patch factorisations), one DC cycle (with_cycle) and one FGMRES
    iteration (a DC cycle plus the Arnoldi step)."""
    from oracle import krylov
    from problems import configs
    from tests.helpers import make_oracle

    if not _C2_PROBLEM:
        _C2_PROBLEM.append(configs.c2())
    pr = _C2_PROBLEM[0]
    prm = dict(configs.TH2D_VANKA)
    t0 = time.perf_counter()
    o = make_oracle(pr, prm)
    t1 = time.perf_counter()
    if with_cycle:
        o.apply(pr.b)
    t2 = time.perf_counter()
    krylov.fgmres(pr.K[0], pr.b, o.apply, rtol=1e-30, restart=30, maxit=1)
    t3 = time.perf_counter()
    return {"setup_s": t1 - t0, "cycle_s": t2 - t1 if with_cycle else None, "iter_s": t3 - t2}


def _oracle_reduced_solve(name):
    """The oracle's FGMRES(30) solve to 1e-8 of a reduced-size config;
    returns its solution with the pressure shifted to zero mean."""
    from oracle import direct, krylov
    from problems import configs
    from tests.helpers import make_oracle

    make, params, note = configs.reduced_cases()[name]
    pr = make()
    t0 = time.perf_counter()
    o = make_oracle(pr, params(pr))
    x, its, rr = krylov.fgmres(pr.K[0], pr.b, o.apply, rtol=1e-8, restart=30, maxit=600)
    t1 = time.perf_counter()
    return {"name": name, "note": note, "iters": its, "true_relres": rr, "seconds": t1 - t0,
            "x": direct.zero_mean_pressure(x, pr.field_off[0], pr.dim, pr.Mp)}


def _pool(workers):
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    return ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))


def _available_gb():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return float(line.split()[1]) / 1e6
    except Exception:
        pass
    return 0.0


def cpu_baseline(solve_iters, reduced=True):
    """The FP64 oracle on the host cores, bounded samples of the C2 solve:
    one process alone (single thread), then as many concurrent single-thread
    processes as cores (capped by memory, about 3 GB each), each timing the
    same sample; plus, when `reduced`, the oracle's full solves of the
    reduced-size configs (their solutions are returned for comparison)."""
    cores = os.cpu_count() or 1
    with _pool(1) as ex:
        one = ex.submit(_oracle_c2_sample).result()
    per_solve = one["setup_s"] + solve_iters * one["iter_s"]
    nproc = max(1, min(cores, int(_available_gb() // 3.5)))
    with _pool(nproc) as ex:
        many = list(ex.map(_oracle_c2_sample, [True] * nproc))
    agg = sum(1.0 / (m["setup_s"] + solve_iters * m["iter_s"]) for m in many)
    out = {"value": 1.0 / per_solve, "unit": "solves/s", "cores": 1, "kind": "oracle",
           "sample": (f"C2: oracle setup ({one['setup_s']:.1f} s), one DC cycle ({one['cycle_s']:.2f} s) and one "
                      f"FGMRES iteration ({one['iter_s']:.2f} s), measured; the solve time is extrapolated to "
                      f"setup + {solve_iters} iterations (the GPU solve's count)"),
           "vcycle_ms": 1e3 * one["cycle_s"], "setup_s": one["setup_s"], "iter_s": one["iter_s"],
           "all_cores": {"value": agg, "unit": "solves/s", "cores": nproc,
                         "sample": f"{nproc} concurrent single-thread processes, each the same sample, extrapolated "
                                   f"the same way; value = sum of their rates",
                         "vcycle_ms_mean": 1e3 * float(np.mean([m["cycle_s"] for m in many]))}}
    if reduced:
        from problems import configs
        names = list(configs.reduced_cases())
        with _pool(min(len(names), cores)) as ex:
            sols = list(ex.map(_oracle_reduced_solve, names))
        out["oracle_solves"] = {r["name"]: {k: v for k, v in r.items() if k != "name"} for r in sols}
        c2 = out["oracle_solves"].get("C2")
        if c2:
            out["measured_solve"] = {"workload": "C2 at 64^2 (the same problem on a 64^2 mesh)", "seconds": c2["seconds"],
                                     "iters": c2["iters"], "cores": 1}
    return out


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores.  Each step is the
    bounded sample of _oracle_c2_sample (oracle setup and one FGMRES
    iteration, single thread, the problem built once before the steps);
    ms_per_step is that measured sample, value the C2 solve rate
    extrapolated from it (setup + ref_iters iterations)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    samples = []
    with _pool(1) as ex:
        for s in range(args.warmup + args.steps):
            r = ex.submit(_oracle_c2_sample, False).result()
            if s >= args.warmup:
                samples.append(r)
    setup = float(np.mean([r["setup_s"] for r in samples]))
    it = float(np.mean([r["iter_s"] for r in samples]))
    step_ms = 1e3 * float(np.mean([r["setup_s"] + r["iter_s"] for r in samples]))
    v = 1.0 / (setup + args.ref_iters * it)
    sample = (f"each step: oracle setup + one FGMRES iteration on C2 (single thread, measured; ms_per_step is "
              f"this sample); value extrapolates a solve as setup + {args.ref_iters} iterations")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "parallelism": "single process, host cores"},
            "value_basis": "extrapolated from the measured per-step sample",
            "iter_ms": 1e3 * it, "setup_ms": 1e3 * setup,
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
def _zero_mean_pressure(pr, x):
    """Shift the pressure to zero mass-weighted mean 1^T Mp p = 0 (the
    solution is unique up to that constant)."""
    off, d = pr.field_off[0], pr.dim
    x = np.array(x, dtype=np.float64)
    p = x[off[d]:off[d + 1]]
    one = np.ones(p.size)
    x[off[d]:off[d + 1]] = p - (one @ (pr.Mp @ p)) / (one @ (pr.Mp @ one))
    return x


def _relerr(a, b):
    """The larger of the 2-norm and the worst-element relative differences."""
    d = a - b
    return float(max(np.linalg.norm(d) / np.linalg.norm(b), np.max(np.abs(d)) / np.max(np.abs(b))))


def _solve_record(sd, torch, pr, prm, prec, stream, reps=2, warm=1, rtol=1e-8, restart=30, maxit=600, cycle=True):
    """Factorisation + FGMRES solve from x0 = 0 timed on the device (CUDA
    events, `reps` steps after `warm`), and the V-cycle alone; returns the
    record and the solution."""
    dev = torch.device("cuda", torch.cuda.current_device())
    h = sd.stokes_setup(pr, dict(prm, precision=prec), stream=stream.cuda_stream)
    b = torch.tensor(pr.b, dtype=torch.float64, device=dev)
    x = torch.zeros_like(b)
    rec = {}
    with torch.cuda.stream(stream):
        def step():
            sd.stokes_factor_patches(h)
            x.zero_()
            return sd.stokes_fgmres_solve(h, b, x, rtol=rtol, restart=restart, maxit=maxit)
        for _ in range(warm):
            rc, info = step()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            rc, info = step()
        e1.record(stream)
        torch.cuda.synchronize()
        iters = [i[0] for i in info]
        rec = {"status": int(rc), "iters": int(max(iters)), "true_relres": float(max(i[2] for i in info)),
               "ms_per_solve": e0.elapsed_time(e1) / reps}
        if len(info) > 1:
            rec["iters_min"] = int(min(iters))
        if cycle:
            z = torch.empty_like(b)
            for _ in range(3):
                sd.stokes_vcycle(h, b, z)
            e0.record(stream)
            for _ in range(10):
                sd.stokes_vcycle(h, b, z)
            e1.record(stream)
            torch.cuda.synchronize()
            rec["vcycle_ms"] = e0.elapsed_time(e1) / 10
            rec["cycle_GBps"] = sd.stokes_cycle_bytes(h) / rec["vcycle_ms"] / 1e6
    xs = x.cpu().numpy()
    sd.stokes_destroy(h)
    return rec, xs


def config_records(sd, torch, stream, c2):
    """Compact records of the other configs (full size, FP32- and
    FP64-preconditioned solves to 1e-8), and the FP32 solutions of the
    reduced-size configs the oracle solves in the cpu_baseline leg."""
    from problems import configs, stokes
    fp32, fp64 = sd.STOKES_FP32, sd.STOKES_FP64
    out = {}

    def both(name, pr, prm, fp64_reps=2, extra=None):
        r32, x32 = _solve_record(sd, torch, pr, prm, fp32, stream)
        r64, x64 = _solve_record(sd, torch, pr, prm, fp64, stream, reps=fp64_reps)
        rec = {"dofs": int(pr.b.size), "levels": int(pr.nlevels), "fp32": r32, "fp64": r64,
               "fp32_vs_fp64_solution_relerr": _relerr(_zero_mean_pressure(pr, x32), _zero_mean_pressure(pr, x64))}
        if extra:
            rec.update(extra(pr, x32))
        out[name] = rec

    def divergence(pr, x):
        off = pr.field_off[0]
        A = pr.K[0][: off[2], : off[2]]
        energy = float(np.sqrt(x[: off[2]] @ (A @ x[: off[2]])))
        return {"divergence_norm_fp32": stokes.divergence_norm(pr, x), "velocity_energy_norm": energy}

    # the setup step of C2 by the host route and by the device route (Alg. 1
    # with the device strength, prolongators, Galerkin products and patch lists)
    from problems import device_setup, mesh as Mh
    setup_s = {}
    for nm, steps in (("host_route_s", stokes.HostSteps), ("device_route_s", device_setup.DeviceSteps(sd))):
        t0 = time.perf_counter()
        stokes.build_th(Mh.unit_square(256), nu=1.0, bc="noslip", rhs="manufactured", max_levels=6, steps=steps)
        torch.cuda.synchronize()
        setup_s[nm] = time.perf_counter() - t0
    out["C2 setup step (mesh, assembly, Alg. 1 hierarchy, patch lists)"] = setup_s
    both("C1 TH2D 16^2 lid, Vanka", configs.c1(), configs.TH2D_VANKA)
    both("C2 TH2D 256^2, DLSC-AMG (DLSC on every level)", c2, configs.th2d_dlsc(c2.nlevels))
    c3 = configs.c3()
    both("C3 SV2D 128^2, Vanka", c3, configs.SV2D_VANKA, extra=divergence)
    both("C3 SV2D 128^2, Vanka on level 0 + DLSC below", c3, configs.sv_vanka_dlsc(c3.nlevels), extra=divergence)
    del c3
    c4 = configs.c4()
    both("C4 TH3D 32^3 lid, stationary Vanka", c4, configs.TH3D_VANKA, fp64_reps=1)
    # FP32 factorisation alone: trailing products of the three-tile-row
    # blocks on mma.sync (default) and on tcgen05
    fac = {}
    for v, nm in ((0, "mma_sync"), (1, "tcgen05")):
        h = sd.stokes_setup(c4, dict(configs.TH3D_VANKA, precision=fp32, factor_tcgen05=v), stream=stream.cuda_stream)
        with torch.cuda.stream(stream):
            sd.stokes_factor_patches(h)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                sd.stokes_factor_patches(h)
            e1.record(stream)
            torch.cuda.synchronize()
        fac[nm] = e0.elapsed_time(e1) / 3
        sd.stokes_destroy(h)
    out["C4 TH3D 32^3 lid, stationary Vanka"]["fp32_factor_ms"] = fac
    kr = dict(schedule=0, nu1=2, nu2=2, eta_u=1.0, eta_p=1.0, omega=1.0,
              relax=[sd.STOKES_RELAX_VANKA_KRYLOV] * (c4.nlevels - 1))
    r, _ = _solve_record(sd, torch, c4, kr, fp32, stream)
    out["C4 TH3D 32^3 lid, Krylov-wrapped Vanka (2 steps per level)"] = {"dofs": int(c4.b.size), "fp32": r}
    del c4
    # the batched workload: all 64 instances in one handle
    probs = configs.c5()
    h = sd.stokes_setup(probs, dict(configs.TH2D_VANKA, precision=fp32), stream=stream.cuda_stream)
    b = torch.tensor(np.concatenate([p.b for p in probs]), dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    with torch.cuda.stream(stream):
        def step():
            sd.stokes_factor_patches(h)
            x.zero_()
            return sd.stokes_fgmres_solve(h, b, x, rtol=1e-8, restart=30, maxit=600)
        step()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        rc, info = step()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    its = [i[0] for i in info]
    out["C5 64 TH2D instances, n ~ U{32..192}, one handle"] = {
        "dofs": int(b.numel()), "instances": len(probs), "instances_per_s": len(probs) * 1000.0 / ms,
        "ms_per_batch": ms, "status": int(rc), "iters_min": int(min(its)), "iters_max": int(max(its)),
        "true_relres_max": float(max(i[2] for i in info))}
    sd.stokes_destroy(h)
    del probs
    # FP32 solutions of the reduced sizes, for the comparison with the oracle
    reduced = {}
    for name, (make, params, note) in configs.reduced_cases().items():
        pr = make()
        _, x32 = _solve_record(sd, torch, pr, params(pr), fp32, stream, reps=1, cycle=False)
        reduced[name] = _zero_mean_pressure(pr, x32)
    return out, reduced


def run_gpu(args):
    import torch

    import paper_2306_06795_gb300 as sd
    from problems import configs

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)

    pr = configs.c2()
    prm = dict(configs.TH2D_VANKA)
    n = pr.b.size
    handles = {}
    for prec in (sd.STOKES_FP32, sd.STOKES_FP64):
        handles[prec] = sd.stokes_setup(pr, dict(prm, precision=prec), stream=stream.cuda_stream)
    h = handles[sd.STOKES_FP32]
    b = torch.tensor(pr.b, dtype=torch.float64, device=dev)
    x = torch.zeros_like(b)
    rtol, restart, maxit = 1e-8, 30, 600

    def step(hh, xx):
        sd.stokes_factor_patches(hh)
        xx.zero_()
        rc, info = sd.stokes_fgmres_solve(hh, b, xx, rtol=rtol, restart=restart, maxit=maxit)
        if rc != sd.STOKES_OK:
            raise RuntimeError(f"solve did not converge: {info}")
        return info[0]

    with torch.cuda.stream(stream):
        # setup-time tuning of the Vanka bins (tiles, ring depth), not timed
        tune = {}
        for prec, hh in handles.items():
            sd.stokes_factor_patches(hh)
            sd.stokes_autotune(hh, 5)
            tune[prec] = json.loads(sd.stokes_autotune_report(hh))
        for _ in range(max(args.warmup, 3)):
            info32 = step(h, x)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        l0 = sd.stokes_kernel_launches(h)
        clocks = ClockSampler(local)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            info32 = step(h, x)
        e1.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        ms = e0.elapsed_time(e1) / args.steps
        launches = (sd.stokes_kernel_launches(h) - l0) // args.steps
        if dist:
            from paper_2306_06795_gb300 import sharding
            ms = sharding.max_over_ranks(ms, dist, device=dev)
            dist.barrier()
        x32 = x.cpu().numpy()

        # FP64-preconditioned form of the same solve
        h64 = handles[sd.STOKES_FP64]
        x64 = torch.zeros_like(b)
        for _ in range(2):
            info64 = step(h64, x64)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        k64 = max(1, args.steps // 2)
        for _ in range(k64):
            info64 = step(h64, x64)
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1) / k64
        x64h = x64.cpu().numpy()

        # the paper's own relaxation for Taylor-Hood (Sec. 3.3.1): Krylov-wrapped,
        # two FGMRES steps with one undamped Vanka sweep each, on every level
        prm_kr = dict(schedule=0, nu1=2, nu2=2, eta_u=1.0, eta_p=1.0, omega=1.0,
                      relax=[sd.STOKES_RELAX_VANKA_KRYLOV] * (pr.nlevels - 1))
        hk = sd.stokes_setup(pr, dict(prm_kr, precision=sd.STOKES_FP32), stream=stream.cuda_stream)
        xk = torch.zeros_like(b)
        for _ in range(2):
            infok = step(hk, xk)
        torch.cuda.synchronize()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        kk = max(1, args.steps // 2)
        for _ in range(kk):
            infok = step(hk, xk)
        g1.record(stream)
        torch.cuda.synchronize()
        msk = g0.elapsed_time(g1) / kk
        zk = torch.empty_like(b)
        for _ in range(3):
            sd.stokes_vcycle(hk, b, zk)
        g0.record(stream)
        for _ in range(10):
            sd.stokes_vcycle(hk, b, zk)
        g1.record(stream)
        torch.cuda.synchronize()
        vck = g0.elapsed_time(g1) / 10
        sd.stokes_destroy(hk)

        # the paper's comparison preconditioner BTP (Sec. 4) on the same solve
        from problems import btp as pbtp
        pr.btp = pbtp.build_btp(pr)
        hb = sd.stokes_setup(pr, dict(prm, precision=sd.STOKES_FP32, preconditioner=sd.STOKES_PRECOND_BTP,
                                      btp_steps=2), stream=stream.cuda_stream)
        xb = torch.zeros_like(b)

        def step_btp():
            xb.zero_()
            rc, info = sd.stokes_fgmres_solve(hb, b, xb, rtol=rtol, restart=restart, maxit=maxit)
            if rc != sd.STOKES_OK:
                raise RuntimeError(f"BTP solve did not converge: {info}")
            return info[0]

        for _ in range(2):
            infob = step_btp()
        torch.cuda.synchronize()
        g0.record(stream)
        for _ in range(kk):
            infob = step_btp()
        g1.record(stream)
        torch.cuda.synchronize()
        msb = g0.elapsed_time(g1) / kk
        sd.stokes_destroy(hb)
        pr.btp = None

        # batched patch factorisation alone
        fct = {}
        for prec, hh in handles.items():
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            for _ in range(3):
                sd.stokes_factor_patches(hh)
            a1.record(stream)
            torch.cuda.synchronize()
            fct[prec] = a0.elapsed_time(a1) / 3

        # V-cycle alone: graph replays, FP32 and FP64
        vc = {}
        r = torch.randn(n, dtype=torch.float64, device=dev, generator=torch.Generator(device=dev).manual_seed(1))
        z = torch.empty_like(r)
        for prec, hh in handles.items():
            for _ in range(5):
                sd.stokes_vcycle(hh, r, z)
            c0 = torch.cuda.Event(enable_timing=True)
            c1 = torch.cuda.Event(enable_timing=True)
            reps = 20
            c0.record(stream)
            for _ in range(reps):
                sd.stokes_vcycle(hh, r, z)
            c1.record(stream)
            torch.cuda.synchronize()
            cms = c0.elapsed_time(c1) / reps
            cb = sd.stokes_cycle_bytes(hh)
            vc[prec] = (cms, cb)

        # dominant kernel: level-0 Vanka gather + patch solve, alone, L2 flushed
        kms, kbytes = sd.stokes_time_kernel(h, sd.STOKES_KERNEL_VANKA_APPLY, 0, reps=20)

        # end to end through the host-pointer entry point (pinned host memory)
        bh = torch.tensor(pr.b, dtype=torch.float64).pin_memory()
        xh = torch.zeros(n, dtype=torch.float64).pin_memory()
        bnp = bh.numpy()
        xnp = xh.numpy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ke = max(1, args.steps // 2)
        for _ in range(ke):
            sd.stokes_factor_patches(h)
            xnp[:] = 0.0
            sd.stokes_fgmres_solve_host(h, bnp, xnp, rtol=rtol, restart=restart, maxit=maxit)
        e2e_s = (time.perf_counter() - t0) / ke
        e2e_res = float(np.linalg.norm(pr.b - pr.K[0] @ xnp) / np.linalg.norm(pr.b))

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peak, peak_kind = measured_peak()
    achieved = kbytes / (kms * 1e-3) / 1e9
    value = ws * 1000.0 / ms
    err32 = float(np.linalg.norm(x32 - x64h) / np.linalg.norm(x64h))
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "dofs": int(n), "levels": int(pr.nlevels),
                   "precision": "FP32 V-cycle, patch factors and applies; FP64 FGMRES, K0 residual, coarsest solve",
                   "step": "stokes_factor_patches + stokes_fgmres_solve from x0 = 0",
                   "l2": "no flush: the cycle's working set (~1 GB) is larger than L2",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "iters": {"fp32": int(info32[0]), "fp64": int(info64[0])},
        "true_relres": {"fp32": float(info32[2]), "fp64": float(info64[2])},
        "fp64_precond": {"value": 1000.0 / ms64, "unit": "solves/s", "ms_per_step": ms64},
        "fp32_vs_fp64_solution_relerr": err32,
        "factor_ms": {"fp32": fct[sd.STOKES_FP32], "fp64": fct[sd.STOKES_FP64]},
        "fgmres": fgmres_leg(int(pr.K[0].shape[0]), int(pr.K[0].nnz), int(info32[0]), 30,
                             (ms - fct[sd.STOKES_FP32] - int(info32[0]) * vc[sd.STOKES_FP32][0]) / int(info32[0]),
                             peak),
        "vcycle": {"fp32_ms": vc[sd.STOKES_FP32][0], "fp64_ms": vc[sd.STOKES_FP64][0],
                   "fp32_bytes": vc[sd.STOKES_FP32][1], "fp64_bytes": vc[sd.STOKES_FP64][1],
                   "fp32_GBps": vc[sd.STOKES_FP32][1] / vc[sd.STOKES_FP32][0] / 1e6,
                   "fp64_GBps": vc[sd.STOKES_FP64][1] / vc[sd.STOKES_FP64][0] / 1e6,
                   "fp32_frac_of_measured_hbm": vc[sd.STOKES_FP32][1] / vc[sd.STOKES_FP32][0] / 1e6 / peak},
        "roofline": {"kernel": "k_vanka_apply_tma (level 0, FP32, 66,049 patches)", "bound": "hbm",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": peak_kind, "traffic": apply_traffic(),
                     "bytes_per_launch": kbytes, "avg_launch_ms": kms},
        "krylov_relax": {"relax": "Krylov-wrapped Vanka (Sec. 3.3.1): 2 FGMRES steps x 1 undamped sweep per level, "
                                  "eta 1, FP32 cycle",
                         "value": 1000.0 / msk, "unit": "solves/s", "ms_per_step": msk, "iters": int(infok[0]),
                         "true_relres": float(infok[2]), "vcycle_ms": vck},
        "btp": {"preconditioner": "block-triangular BTP (Sec. 4): SA V-cycle on A, SA V-cycle on M_p/nu, "
                                  "2 Krylov-wrapped Jacobi steps, FP32 cycles",
                "value": 1000.0 / msb, "unit": "solves/s", "ms_per_step": msb, "iters": int(infob[0]),
                "true_relres": float(infob[2]),
                "dc_solve_ms_without_factorisation": ms - fct[sd.STOKES_FP32],
                "dc_solve_time_over_btp": (ms - fct[sd.STOKES_FP32]) / msb if msb > 0 else None},
        "e2e": {"value": 1.0 / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": int(16 * n),
                "d2h_bytes_per_step": int(8 * n), "true_relres": e2e_res},
        "autotune_fp32": tune[sd.STOKES_FP32]["bins"],
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if ws == 1 and args.configs:
        with torch.cuda.stream(stream):
            # the paper's own solver setting (Sec. 4): FGMRES(20), residual reduced by 1e10
            ps = {}
            for prec, nm in ((sd.STOKES_FP32, "fp32"), (sd.STOKES_FP64, "fp64")):
                ps[nm], _ = _solve_record(sd, torch, pr, prm, prec, stream, rtol=1e-10, restart=20, cycle=False)
            line["paper_setting"] = {"solver": "FGMRES(20) to a 1e-10 relative residual (Sec. 4)", **ps}
            recs, reduced = config_records(sd, torch, stream, pr)
        line["configs"] = recs
    if args.cpu_baseline and ws == 1:
        cb = cpu_baseline(int(info32[0]), reduced=args.configs)
        solves = cb.pop("oracle_solves", {})
        fp32_vs_oracle = {}
        for name, r in solves.items():
            if args.configs and name in reduced:
                fp32_vs_oracle[name] = {"relerr": _relerr(reduced[name], r["x"]), "at": r["note"],
                                        "oracle_iters": r["iters"]}
        if fp32_vs_oracle:
            line["fp32_vs_oracle_solution"] = fp32_vs_oracle
        line["cpu_baseline"] = cb
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_profile(args):
    """Kernel launches for ncu: factorisation, then DC cycles (graph replays),
    on C2 (default), C2 with DLSC relaxation on every level (`c2-dlsc`), C4,
    or the 3D Taylor-Hood lid-driven cavity on an N^3 cube (`cubeN`, a small
    case of the C4 kernels)."""
    import torch

    import paper_2306_06795_gb300 as sd
    from problems import configs, mesh, stokes

    name = args.profile_problem or "c2"
    if name == "c2":
        pr, prm = configs.c2(), configs.TH2D_VANKA
    elif name == "c2-dlsc":
        pr = configs.c2()
        prm = configs.th2d_dlsc(pr.nlevels)
    elif name == "c4":
        pr, prm = configs.c4(), configs.TH3D_VANKA
    else:
        pr, prm = stokes.build_th(mesh.unit_cube(int(name[4:])), bc="lid"), configs.TH3D_VANKA
    stream = torch.cuda.Stream()
    h = sd.stokes_setup(pr, dict(prm, precision=sd.STOKES_FP32), stream=stream.cuda_stream)
    sd.stokes_factor_patches(h)
    r = torch.tensor(pr.b, dtype=torch.float64, device="cuda")
    z = torch.empty_like(r)
    for _ in range(args.profile_cycles):
        sd.stokes_vcycle(h, r, z)
    if args.profile_solve:
        with torch.cuda.stream(stream):
            sd.stokes_fgmres_solve(h, r, z.zero_(), rtol=1e-8, restart=30, maxit=600)
    torch.cuda.synchronize()


def run_gpu_c5(args):
    """The batched workload (64 Taylor-Hood instances of different sizes and
    viscosities): each rank solves its DoF-balanced share of the instances
    in one handle (no data-path collective); value = instances solved per
    second over all ranks, timed as the maximum over ranks."""
    import torch

    import paper_2306_06795_gb300 as sd
    from paper_2306_06795_gb300 import sharding
    from problems import configs

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    inst = configs.c5_instances()
    dofs = [2 * (2 * n + 1) ** 2 + (n + 1) ** 2 for n, _, _ in inst]
    mine = sharding.shard_instances(dofs, ws)[rank]
    probs = configs.c5()
    probs = [probs[i] for i in mine]
    h = sd.stokes_setup(probs, dict(configs.TH2D_VANKA, precision=sd.STOKES_FP32), stream=stream.cuda_stream)
    b = torch.tensor(np.concatenate([p.b for p in probs]), dtype=torch.float64, device=dev)
    x = torch.zeros_like(b)

    def step():
        sd.stokes_factor_patches(h)
        x.zero_()
        rc, info = sd.stokes_fgmres_solve(h, b, x, rtol=1e-8, restart=30, maxit=600)
        if rc != sd.STOKES_OK:
            raise RuntimeError(f"batched solve did not converge: {info}")
        return info

    with torch.cuda.stream(stream):
        sd.stokes_factor_patches(h)
        sd.stokes_autotune(h, 5)
        for _ in range(max(args.warmup, 3)):
            info = step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        l0 = sd.stokes_kernel_launches(h)
        clocks = ClockSampler(local)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            info = step()
        e1.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        ms = sharding.max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, device=dev)
        launches = (sd.stokes_kernel_launches(h) - l0) // args.steps
    if rank == 0:
        its = [i[0] for i in info]
        line = {"metric": "Stokes instances solved/s to 1e-8 rel-res (batched, FP32 DC-AMG preconditioned FGMRES)",
                "value": len(inst) * 1000.0 / ms, "unit": "instances/s", "n_gpus": ws, "steps": args.steps,
                "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "64 x 2D Taylor-Hood P2/P1, n ~ U{32..192}, nu = 10^U(-2,2), random b, "
                                       "no slip; all instances of a rank in one handle",
                           "dofs": int(sum(dofs)), "instances_rank0": len(mine),
                           "parallelism": f"instance shards over {ws} GPU(s)"},
                "iters": {"min": int(min(its)), "max": int(max(its))}, "gpu_launches": int(launches),
                "clocks": clk}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-configs", dest="configs", action="store_false",
                    help="skip the per-config records and the paper-setting record of the default line")
    ap.add_argument("--profile-cycles", type=int, default=0,
                    help="profiling driver: set up, factorise and run this many DC cycles, print nothing")
    ap.add_argument("--profile-problem", default=None,
                    help="profiling driver problem: c2 (default), c2-dlsc, c4, or cubeN (3D lid-driven cavity on an N^3 cube)")
    ap.add_argument("--profile-solve", action="store_true",
                    help="profiling driver: set up, factorise and run one FP32-preconditioned solve")
    ap.add_argument("--ref-iters", type=int, default=34,
                    help="iterations a full oracle solve takes (scales the reference sample)")
    ap.add_argument("--workload", default="c2", choices=["c2", "c5"],
                    help="c2: the single 256^2 problem (default); c5: the 64-instance batch, sharded over ranks")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.profile_cycles or args.profile_solve or args.profile_problem:
        run_profile(args)
    elif args.workload == "c5":
        run_gpu_c5(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
