"""Write the stored oracle trajectories under tests/golden/ (calls only oracle/ and the
seeded input generators).

    python -m tests.golden.make_golden
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import wcsph as o                                  # noqa: E402
from paper_2010_12375_gb300 import workloads as wk             # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def dam_break_2d_trajectory():
    prob = wk.dam_break_2d()                 # H = 1, L = 2, dp = H/40, t_end = 5 sqrt(H/g)
    _, series = o.run(prob)
    tank = wk.TANK_EXTENT * prob.meta["H"]
    t_impact = next((s["t"] for s in series if s["front_x"] >= tank - 2 * prob.dp), None)
    out = {
        "_source": "oracle/wcsph.py run of paper_2010_12375_gb300.workloads.dam_break_2d() "
                   "(2D dam break, 3200 fluid particles) to t = 5 sqrt(H/g); one record per "
                   "advection step",
        "t_end": prob.t_end,
        "t_impact": t_impact,
        "t": [s["t"] for s in series],
        "energy": [s["energy"] for s in series],
        "kinetic": [s["kinetic"] for s in series],
        "potential": [s["potential"] for s in series],
        "internal": [s["internal"] for s in series],
        "front_x": [s["front_x"] for s in series],
        "substeps": [s["substeps"] for s in series],
    }
    with open(os.path.join(HERE, "dam_break_2d_trajectory.json"), "w") as f:
        json.dump(out, f)
    return out


def sloshing_centre_of_mass():
    """The sloshing tank (L = 1, d = 0.5, dp = 0.02) in its own frame: a horizontal pulse of
    the tank's acceleration (body force -0.05 g along x for t < 0.1) and then free sloshing;
    the fluid's mean x after every advection step from t = 0.1 to 4.5 linear periods."""
    import copy
    import numpy as np
    prob = wk.sloshing_tank(L=1.0, d=0.5, dp=0.02)
    g = prob.meta["g"]
    pulse = copy.copy(prob)
    pulse.gravity = np.array([-0.05 * g, -g, 0.0])
    prm_pulse, prm_free = o.Params.from_problem(pulse), o.Params.from_problem(prob)
    st, w = o.state_from_problem(prob)
    t, x = [], []
    while st.t < 4.5 * prob.meta["period_1"]:
        st, _ = o.advection_step(st, w, prm_pulse if st.t < 0.1 else prm_free)
        if st.t >= 0.1:
            t.append(st.t)
            x.append(float(np.mean(st.x[:, 0])))
    out = {
        "_source": "oracle/wcsph.py run of paper_2010_12375_gb300.workloads.sloshing_tank(L=1, d=0.5, "
                   "dp=0.02), gravity (-0.05 g, -g) while t < 0.1 then (0, -g), switched between "
                   "advection steps; the fluid's mean x after each advection step from t = 0.1",
        "period_linear": prob.meta["period_1"],
        "t": t,
        "x_mean": x,
    }
    with open(os.path.join(HERE, "sloshing_tank_com.json"), "w") as f:
        json.dump(out, f)
    return out


if __name__ == "__main__":
    which = sys.argv[1:] or ["dam_break", "sloshing"]
    if "dam_break" in which:
        d = dam_break_2d_trajectory()
        print(len(d["t"]), d["t_impact"], d["energy"][0], d["energy"][-1], d["substeps"][-1])
    if "sloshing" in which:
        d = sloshing_centre_of_mass()
        print(len(d["t"]), d["period_linear"])
