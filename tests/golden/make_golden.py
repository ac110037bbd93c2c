"""Write the oracle-derived regression fixtures in this folder.

Calls only ``oracle`` (never the CUDA library).  Run from the repository root:
``python tests/golden/make_golden.py``.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402


def main():
    consts = json.load(open(os.path.join(HERE, "paper_constants.json")))
    x = np.array(consts["toy_dataset"]["x"], dtype=np.float64)
    h = oracle.grid_log(0.05, 2.0, 16)
    r = oracle.lscv_h(x, h)
    p = oracle.plugin(x)
    out = {
        "_about": "Oracle values for the paper's 8-point toy set (Sec. 4.2). "
                  "Regression fixture written by make_golden.py; not a paper pin.",
        "h": h.tolist(),
        "g": r["g"].tolist(),
        "argmin": r["argmin"],
        "plugin": {k: p[k] for k in ("sigma", "g1", "psi6", "g2", "psi4", "h")},
        "plugin_status": p["status"],
    }
    with open(os.path.join(HERE, "toy8_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
