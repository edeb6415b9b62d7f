"""Host logic of bench.py that needs no GPU: the clock record counts only
the nvidia-smi samples taken inside the timed region and reports every
throttle reason seen there."""
import os

import bench


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler(path, lines, skip):
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")
    c = bench.ClockSampler.__new__(bench.ClockSampler)
    c.path = str(path)
    c.f = open(os.devnull, "w")
    c.proc = _Proc()
    c.skip = skip
    return c


def test_samples_before_the_timed_region_are_skipped(tmp_path):
    idle = "345, 2070, 120.5, 0x1, Not Active, Not Active, Not Active, Not Active"
    busy = "2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active"
    capped = "1980, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active"
    rec = _sampler(tmp_path / "c.csv", [idle, busy, busy, capped], skip=1).stop()
    assert rec["samples"] == 3
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]


def test_thermal_slowdown_is_reported(tmp_path):
    hot = "1500, 2070, 1000.0, 0x40, Not Active, Active, Not Active, Not Active"
    rec = _sampler(tmp_path / "c.csv", [hot, hot], skip=0).stop()
    assert rec["reasons"] == ["hw_thermal_slowdown"] and rec["samples"] == 2


def test_no_samples(tmp_path):
    rec = _sampler(tmp_path / "c.csv", ["garbage"], skip=0).stop()
    assert rec["reasons"] == ["no samples"]


def test_sampler_without_nvidia_smi_reports_unavailable():
    """Constructing the sampler never fails; without nvidia-smi (this
    container) the record says so."""
    import shutil
    c = bench.ClockSampler(0)
    rec = c.stop()
    if shutil.which("nvidia-smi") is None:
        assert rec["reasons"] == ["nvidia-smi unavailable"]


def test_roofline_traffic_is_null_unless_the_kernel_sources_match(monkeypatch):
    import hashlib
    h = hashlib.sha256()
    for f in bench.APPLY_L0_TRAFFIC["sources"]:
        with open(os.path.join(bench.ROOT, "paper_2306_06795_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    rec = dict(bench.APPLY_L0_TRAFFIC)
    monkeypatch.setattr(bench, "APPLY_L0_TRAFFIC", dict(rec, sha256=h.hexdigest()))
    assert bench.apply_traffic() == rec["dram_bytes"]
    monkeypatch.setattr(bench, "APPLY_L0_TRAFFIC", dict(rec, sha256="0" * 64))
    assert bench.apply_traffic() is None


def test_relerr_takes_the_worst_element():
    import numpy as np
    b = np.ones(10000)
    a = b.copy()
    a[3] += 1e-4
    assert bench._relerr(a, b) == pytest_approx(1e-4)


def test_zero_mean_pressure_removes_the_mass_weighted_mean():
    import numpy as np
    from problems import configs
    pr = configs.c1()
    x = np.random.default_rng(0).standard_normal(pr.b.size)
    y = bench._zero_mean_pressure(pr, x)
    off = pr.field_off[0]
    p = y[off[2]:off[3]]
    assert abs(np.ones(p.size) @ (pr.Mp @ p)) < 1e-12 * np.abs(p).sum()
    assert np.array_equal(y[: off[2]], x[: off[2]])


def pytest_approx(v):
    import pytest
    return pytest.approx(v, rel=1e-9)


def test_fgmres_leg_counts_the_arnoldi_steps_of_each_restart():
    """Iterations 1..3 with restart 2 use 1, 2, then 1 basis vectors; each
    step reads K0 once (12 B per nonzero) and V in three passes."""
    import bench
    n, nnz = 10, 30
    rec = bench.fgmres_leg(n, nnz, 3, 2, 0.5, 1000.0)
    per = [nnz * 12 + 4 * (n + 1) + 16 * n + (3 * k + 5) * 8 * n + 20 * n for k in (1, 2, 1)]
    assert rec["bytes_per_iter"] == sum(per) / 3
    assert rec["dfma_per_iter"] == sum(nnz + (4 * k + 1) * n for k in (1, 2, 1)) / 3
    assert abs(rec["GBps"] - rec["bytes_per_iter"] / 0.5 / 1e6) < 1e-12
    assert abs(rec["frac_of_measured_hbm"] - rec["GBps"] / 1000.0) < 1e-12
