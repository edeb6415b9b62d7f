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
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
