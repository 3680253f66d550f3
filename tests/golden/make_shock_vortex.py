"""Writes shock_vortex.json: the set-up of the shock-vortex interaction (Sec. IV H) for the ideal
gas and the BZT van der Waals gas, computed by the oracle's set-up routines
(oracle/shock_vortex.py) and nothing else.

Per configuration: the EOS, domain, grid, shock position, vortex parameters and end time the
paper states; the upstream state (rho1, u1 = M_s c_s1, P1) and the exact downstream state of the
stationary normal shock; and the vortex's radial profile rho(r), P(r) on r = j dr, sampled from an
RK2 integration along the ambient isentrope (stored to r = 7, beyond which it equals the ambient
state to 1e-12).

    python tests/golden/make_shock_vortex.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import shock_vortex as SV  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "shock_vortex.json")
DR, R_KEEP, FINE = 0.01, 7.0, 100  # stored spacing, stored extent, integration substeps per DR

CONFIGS = {
    # Sec. IV H, ideal gas: gamma 1.4, ambient rho1 = 1, P1 = 1; t_end = 7 at 800 x 300
    "ideal": {"eos": {"kind": "ideal", "gamma": 1.4}, "rho1": 1.0, "P1": 1.0, "grid": [800, 300], "t_end": 7.0},
    # Sec. IV H, BZT: the van der Waals gas of Sec. IV F (a = 1, b = 0.3, R = 1, gamma = 1 + R/cv = 1.02),
    # ambient rho1 = 0.70 and the printed P1 = 0.3787 (T1 ~ 0.980); t_end = 15 at 1200 x 450
    "bzt": {"eos": {"kind": "vdw", "a": 1.0, "b": 0.3, "R": 1.0, "cv": 50.0}, "rho1": 0.70, "P1": 0.3787,
            "grid": [1200, 450], "t_end": 15.0},
}


def make():
    out = {"cite": "Sec. IV H", "domain": [0.0, 16.0, 0.0, 6.0], "x_shock": 6.0, "vortex_centre": [2.0, 3.0],
           "beta_v": 2.0, "Rc": 1.0, "Ms": 1.2, "profile_dr": DR}
    for name, c in CONFIGS.items():
        up, down = SV.normal_shock(c["eos"], c["rho1"], c["P1"], 1.2)
        n = int(round(12.0 / DR)) * FINE
        r, rho, e, P = SV.vortex_profile(c["eos"], up[0], up[2], beta_v=2.0, Rc=1.0, r_max=12.0, n=n)
        keep = int(round(R_KEEP / DR))
        out[name] = {"eos": c["eos"], "grid": c["grid"], "t_end": c["t_end"], "upstream": list(up),
                     "downstream": list(down),
                     "profile_rho": [float(x) for x in rho[: keep * FINE + 1: FINE]],
                     "profile_P": [float(x) for x in P[: keep * FINE + 1: FINE]]}
    return out


if __name__ == "__main__":
    with open(OUT, "w") as fh:
        json.dump(make(), fh, indent=1)
    print(OUT)
