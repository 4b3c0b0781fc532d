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


if __name__ == "__main__":
    d = dam_break_2d_trajectory()
    print(len(d["t"]), d["t_impact"], d["energy"][0], d["energy"][-1], d["substeps"][-1])
