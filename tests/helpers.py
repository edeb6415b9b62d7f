"""Shared test helpers: oracle construction from a workload's parameters."""
import numpy as np

from oracle import cycle


def oracle_params(pr, prm):
    nrel = pr.nlevels - 1
    om = prm.get("omega", 1.0)
    omega = [float(om)] * nrel if np.isscalar(om) else list(om)
    if "omega0" in prm:
        omega[0] = prm["omega0"]
    return cycle.Params(schedule=prm.get("schedule", 0), nu1=prm.get("nu1", 1), nu2=prm.get("nu2", 1),
                        eta_u=prm.get("eta_u", 1.0), eta_p=prm.get("eta_p", 1.0), omega=omega,
                        relax=prm.get("relax"),
                        cheb_deg=prm.get("cheb_deg", (3, 3, 6) if pr.dim == 2 else (4, 4, 16)),
                        mcg_deg=prm.get("mcg_deg", 32), dlsc_sweeps=prm.get("dlsc_sweeps", 2))


def make_oracle(pr, prm):
    return cycle.Oracle(pr, oracle_params(pr, prm))


def rel(a, b):
    """Relative difference of a against the reference b, the larger of the
    2-norm ratio ||a - b|| / ||b|| and the worst-element ratio
    max|a - b| / max|b|: a wrong value confined to a few entries cannot hide
    under a whole-vector norm."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if a.shape != b.shape:
        raise ValueError(f"shapes differ: {a.shape} vs {b.shape}")
    if a.size == 0:
        return 0.0
    d = a - b
    two = np.linalg.norm(d) / max(np.linalg.norm(b), 1e-300)
    worst = np.max(np.abs(d)) / max(np.max(np.abs(b)), 1e-300)
    return float(max(two, worst))
