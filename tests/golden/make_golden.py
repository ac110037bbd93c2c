"""Write the oracle-derived regression fixtures in this folder.

Calls only ``oracle`` and the seeded input generators (never the CUDA
library).  Run from the repository root: ``python tests/golden/make_golden.py``
(toy set), ``python tests/golden/make_golden.py --full-skewed`` (the full
n = 65,536 skewed-column oracle; minutes on a multi-core host) and
``python tests/golden/make_golden.py --full-mixture`` (the full n = 16,384,
d = 2, 3, 4 correlated-mixture oracle; minutes).
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


def full_correlated_mixture():
    """The full oracle of the multivariate LSCV selection: n = 16,384 samples of
    the 4-component correlated mixture (datagen.correlated_mixture(n, d,
    seed=3+d)) for d = 2, 3, 4, H = h^2 S on the 128-point grid over Z(h0):
    g(h), both exponential sums and the argmin over all 1.3e8 pairs, in FP64
    (Sec. 4.4.2, Eqs. LSCV-gh, LSCV-Kx, LSCV-KKx)."""
    from paper_1505_01998_gb300 import datagen
    n, n_h = 16384, 128
    out = {
        "_about": "FP64 oracle over all pairs of the n = 16,384 correlated mixtures "
                  "(datagen.correlated_mixture(16384, d, seed=3+d), d = 2, 3, 4): LSCV with "
                  "H = h^2 S, g(h), its exponential sums and argmin on the 128-point grid over "
                  "Z(h0). Written by make_golden.py --full-mixture; calls only the oracle.",
        "n": n, "n_h": n_h, "cases": {},
    }
    for d in (2, 3, 4):
        x = datagen.correlated_mixture(n, d, seed=3 + d).astype(np.float64)
        h = oracle.grid_default(n, d, n_h)
        r = oracle.lscv_h(x, h)
        out["cases"][str(d)] = {"seed": 3 + d, "h": h.tolist(), "g": r["g"].tolist(),
                                "s_kk": r["s_kk"].tolist(), "s_k": r["s_k"].tolist(),
                                "argmin": r["argmin"]}
    with open(os.path.join(HERE, "mixture16384_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)


def main():
    if "--full-skewed" in sys.argv:
        full_skewed_column()
        return
    if "--full-mixture" in sys.argv:
        full_correlated_mixture()
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
