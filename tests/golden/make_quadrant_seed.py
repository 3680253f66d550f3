"""Writes quadrant_seed.json: the seed of the 2D four-quadrant Riemann input (ideal gas,
gamma 1.4, quadrant states rho~U[0.1,2], u,v~U[-1,1], P~U[0.05,2], zero-gradient boundaries,
CFL 0.5, sensor B with beta_min 0.75, C_sensor 4) and its states.  The seed is the first one,
counting up from 2, whose oracle run on a 512 x 512 copy stays physical (rho > 0, c_s^2 > 0) up
to t = 0.25.  Many random quadrant states do not: with the stated sensor constants the
method turns non-physical within a few hundred steps (near-vacuum states, or grid-scale growth
where the sensor leaves beta near 1).  Calls only the oracle and the input generator.

    python tests/golden/make_quadrant_seed.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2609_10639_b300 import workloads as wl  # noqa: E402


def survives(seed, n=512):
    """(reached t_end, time reached, steps taken) of the oracle run of this seed's states."""
    p = wl.QUADRANTS_2D.resized(n)
    s = O.OracleSolver.for_problem(p)
    s.init(wl.quadrants_2d(p, seed=seed))
    try:
        s.step(10 ** 7, p.t_end)
    except ValueError:
        pass
    t, steps, _ = s.time()
    return t == p.t_end, t, steps


def main():
    tried = []
    for seed in range(2, 40):
        ok, t, steps = survives(seed)
        tried.append({"seed": seed, "ok": bool(ok), "t_reached": t, "steps": steps})
        print(seed, ok, t, steps, flush=True)
        if ok:
            out = {"seed": seed, "states_NE_NW_SW_SE": [list(s) for s in wl.quadrant_states(seed)],
                   "rule": "first seed >= 2 whose oracle run at 512x512 stays physical to t = 0.25",
                   "tried": tried}
            path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "quadrant_seed.json")
            with open(path, "w") as fh:
                json.dump(out, fh, indent=1)
                fh.write("\n")
            return
    raise SystemExit("no seed accepted")


if __name__ == "__main__":
    main()
