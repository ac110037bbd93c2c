"""Write the oracle-derived regression fixtures in this folder.

Calls only ``oracle`` and the seeded input generators (never the CUDA
library).  Run from the repository root: ``python tests/golden/make_golden.py``
(toy set) and ``python tests/golden/make_golden.py --full-skewed`` (the full
n = 65,536 skewed-column oracle; minutes on a multi-core host).
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402


def full_skewed_column():
    """The full oracle of the n = 65,536 skewed-column selection (LSCV_h on the
    256-point grid over Z(h0) and the PLUGIN chain): every one of the 2.1e9
    pairs, in FP64.  Minutes on a multi-core host."""
    from paper_1505_01998_gb300 import datagen
    n = 65536
    x = datagen.skewed_column(n, seed=2).astype(np.float64)  # the FP32 values the device sees
    h = oracle.grid_default(n, 1, 256)
    r = oracle.lscv_h(x, h)
    p = oracle.plugin(x)
    out = {
        "_about": "FP64 oracle over all pairs of the n = 65,536 skewed column "
                  "(datagen.skewed_column(65536, seed=2)): LSCV_h g(h), its exponential sums "
                  "and argmin on the 256-point grid over Z(h0), and the PLUGIN chain. "
                  "Written by make_golden.py --full-skewed; calls only the oracle.",
        "n": n, "seed": 2,
        "h": h.tolist(), "g": r["g"].tolist(), "s_kk": r["s_kk"].tolist(), "s_k": r["s_k"].tolist(),
        "argmin": r["argmin"],
        "plugin": {k: p[k] for k in ("sigma", "g1", "psi6", "g2", "psi4", "h")},
        "plugin_status": p["status"],
    }
    with open(os.path.join(HERE, "skewed65536_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)


def main():
    if "--full-skewed" in sys.argv:
        full_skewed_column()
        return
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
