"""Writes bzt_states_seed3.json: the left/right (rho, P) states of the 2D BZT interface problem
(reduced van der Waals units a = 3, b = 1/3, R = 8/3, cv = 50 R).  Candidates are drawn from the
seeded stream of the input generator; a candidate is kept only where the oracle's EOS gives
c_s^2 > 0 and fundamental derivative Gamma < 0, and a pair of kept states only if the oracle's
run of the interface problem they start (128 x 128 copy, to t = 0.2) stays hyperbolic, c_s^2 > 0
throughout the states the flow visits (Eq. 14).  Subcritical states near the spinodal pass the
first test but are driven to c_s^2 < 0 within a few steps by the expansion wave.  Calls only the
oracle and the input generator.

    python tests/golden/make_bzt_states.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2609_10639_b300 import workloads as wl  # noqa: E402


def accept(rho, P, eos=wl.VDW_REDUCED):
    e = wl.internal_energy(eos, rho, P)
    _, cs2 = O.eos_eval(eos, rho, e)
    return cs2 > 0.0 and O.fundamental_derivative(eos, rho, e) < 0.0


def pair_ok(left, right, n=128):
    p = wl.BZT_2D.resized(n)
    s = O.OracleSolver.for_problem(p)
    s.init(wl.bzt_interface_2d(p, states=[left, right]))
    try:
        s.step(10 ** 6, p.t_end)
    except ValueError:
        return False
    return s.time()[0] == p.t_end


def main(seed=3):
    left, right = wl.bzt_states(seed, accept=accept, pair_ok=pair_ok)
    out = {"seed": seed, "eos": wl.VDW_REDUCED, "left": list(left), "right": list(right),
           "rule": "first pair of consecutive kept candidates (c_s^2 > 0 and Gamma < 0, oracle EOS) whose "
                   "oracle run at 128x128 to t = 0.2 stays hyperbolic"}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"bzt_states_seed{seed}.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")
    print(path, out)


if __name__ == "__main__":
    main()
