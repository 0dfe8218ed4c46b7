"""Writes config1_oracle.json: the oracle's loop on the 60x20x4 cantilever.

The paper's usage example (Section 3) and benchmark (Section 4.2) are
cantilevers of this kind; the paper prints no iteration history, so the
stored values are the oracle's own (this script calls only ``oracle`` and
the input generators).  Bisection runs to 1e-12 so that the volume is on
target to 1e-6 (with the customary 1e-3 it is only within ~1e-4).

    python tests/golden/make_config1.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import topopt  # noqa: E402
from synth import problems  # noqa: E402

ITERS = 50
BISECT_TOL = 1e-12


def main():
    prob = problems.config_small(iters=ITERS)
    prob.bisect_tol = BISECT_TOL
    x, hist = topopt.top3d(prob, solver="direct")
    out = {
        "source": "oracle.topopt.top3d, direct solves, tests/golden/make_config1.py",
        "problem": {"nelx": prob.nelx, "nely": prob.nely, "nelz": prob.nelz,
                    "volfrac": prob.volfrac, "penal": prob.penal, "rmin": prob.rmin,
                    "load": "unit -y on the nodes of the x=nelx, y=0 edge", "clamped": "x=0 face",
                    "bisect_tol": BISECT_TOL, "iters": ITERS},
        "compliance": [h.compliance for h in hist],
        "volume": [h.volume for h in hist],
        "halvings": [h.halvings for h in hist],
        "final_compliance_check": hist[-1].compliance,
    }
    with open(os.path.join(HERE, "config1_oracle.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
