"""Writes tests/golden/bubbles_400m.json: the FP64 oracle's state of the two
validation cases of Sec. 3 at 400 m resolution, summarised by
tests/bubble_diag.py -- the density current at 900 s and the rising bubble
at 1000 s (the times of the paper's figures).  Calls only oracle/ and the
input builders.  Run from the repository root:

    python tests/golden/make_bubbles.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

from bubble_diag import bubble_diagnostics  # noqa: E402
from oracle import Oracle  # noqa: E402
from paper_2301_04698_gb300 import inputs  # noqa: E402

CASES = {"density_current": (inputs.density_current, 900.0), "rising_bubble": (inputs.rising_bubble, 1000.0)}


def main():
    out = {"source": "FP64 oracle (oracle/), tests/golden/make_bubbles.py", "dx_m": 400.0, "cases": {}}
    for name, (builder, t_end) in CASES.items():
        c = builder(400.0)
        o = Oracle(c, inputs.initial_state(c))
        steps = int(round(t_end / c.dt))
        o.step(steps)
        d = bubble_diagnostics(c, o.get("theta_l"), o.get("u"), o.get("w"))
        out["cases"][name] = {"t_s": t_end, "steps": steps, **d}
        print(name, d, flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "bubbles_400m.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
