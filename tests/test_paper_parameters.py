"""The workload configurations and the DLSC defaults use the parameters the
paper prints (tests/golden/paper_tables.json, each entry with its table):
Chebyshev degrees and interval of DLSC (Table lsd_dgs_config), the optimal
eta of the Taylor-Hood DC-all Vanka and DLSC preconditioners (Table p2p1_taus) and the
optimal (omega_0, eta_p) of the Scott-Vogelius ones (Table p2p1disc_params)."""
import json
import os

from oracle import dlsc
from problems import configs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_tables.json")


def tables():
    with open(GOLDEN) as f:
        return json.load(f)


def test_taylor_hood_eta_is_the_dc_all_optimum():
    t = tables()["taylor_hood_eta_opt"]
    assert configs.TH2D_VANKA["schedule"] == 0  # DC-all
    assert configs.TH2D_VANKA["eta_u"] == configs.TH2D_VANKA["eta_p"] == t["vanka_dc_all_2d"]
    assert configs.TH3D_VANKA["eta_u"] == configs.TH3D_VANKA["eta_p"] == t["vanka_dc_all_3d"]


def test_taylor_hood_dlsc_eta_is_the_dc_all_optimum():
    t = tables()["taylor_hood_eta_opt_dlsc"]
    v = configs.th2d_dlsc(6)
    assert v["schedule"] == 0 and v["eta_u"] == v["eta_p"] == t["dlsc_dc_all_2d"]
    assert v["relax"] == [1] * 5 and v["dlsc_sweeps"] == 2  # DLSC on every level, two sweeps


def test_scott_vogelius_parameters_are_the_structured_optimum():
    t = tables()["scott_vogelius_structured"]
    assert (configs.SV2D_VANKA["omega0"], configs.SV2D_VANKA["eta_p"]) == (t["vanka"]["omega0"], t["vanka"]["eta_p"])
    v = configs.sv_vanka_dlsc(5)
    assert (v["omega0"], v["eta_p"]) == (t["vanka_level0_dlsc_coarse"]["omega0"],
                                         t["vanka_level0_dlsc_coarse"]["eta_p"])
    assert v["relax"] == [0, 1, 1, 1]  # Vanka on level 0, DLSC on the coarser levels


def test_dlsc_defaults_follow_the_chebyshev_table():
    t = tables()["dlsc_chebyshev_degrees"]
    import paper_2306_06795_gb300 as sd
    for dim, key in ((2, "2d"), (3, "3d")):
        s = sd._params(sd._Keep(), {}, 3, dim)
        assert tuple(s.cheb_deg) == tuple(t[key])
        assert tuple(sd.DLSC_DEGREES[dim]) == tuple(t[key])


def test_oracle_dlsc_uses_the_chebyshev_interval(monkeypatch):
    """Each DLSC stage runs a Chebyshev iteration on [0.5^d lambda, 1.1 lambda]
    with lambda the estimate of the stage's operator."""
    import numpy as np
    import scipy.sparse as sp
    t = tables()["dlsc_chebyshev_interval"]
    seen = []

    def record(op, b, lo, hi, degree, dinv=None):
        seen.append((lo, hi, degree))
        return np.zeros_like(b)

    monkeypatch.setattr(dlsc, "chebyshev", record)

    class Prob:
        dim = 3
        K = [sp.identity(5, format="csr")]
        field_off = [np.array([0, 1, 2, 3, 5])]
        lambda_A = [2.0]
        lambda_S = [8.0]
        Mu_diag = np.ones(3)

    class Par:
        cheb_deg = (4, 4, 16)
        dlsc_sweeps = 1

    lev = dlsc.DLSCLevel(Prob(), 0, Par())
    lev.one(np.zeros(5), np.ones(5))
    lo3 = t["lower_base"] ** 3
    assert seen == [(lo3 * 2.0, t["upper_factor"] * 2.0, 4), (lo3 * 8.0, t["upper_factor"] * 8.0, 4),
                    (lo3 * 8.0, t["upper_factor"] * 8.0, 16)]
