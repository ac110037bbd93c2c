"""Write the oracle-derived regression fixtures in this folder.

Calls only ``oracle`` and the seeded input generators (never the CUDA
library).  Run from the repository root: ``python tests/golden/make_golden.py``
(toy set), ``python tests/golden/make_golden.py --full-skewed`` (the full
n = 65,536 skewed-column oracle; minutes on a multi-core host) and
``python tests/golden/make_golden.py --full-mixture`` (the full n = 16,384,
d = 2, 3, 4 correlated-mixture oracle; minutes) and
``python tests/golden/make_golden.py --batch`` (the 512-dataset batch: the
full oracle of every dataset with n <= 16,384 and of the 16 smallest above;
about an hour on 8 host cores).
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


def batch_subset():
    """The full oracle of the batched workload's datasets (datagen.batch(512,
    seed=4): sizes log-uniform on [256, 131072], each a 1-5 component mixture
    or a lognormal): every dataset with n <= 16,384 and the 16 smallest above
    it, each LSCV_h on the 128-point grid over Z(h0) (Sec. 4.4.2, Eq.
    LSCV-Zh0) and the PLUGIN chain (Sec. 4.4.1).  Stored per dataset: the
    argmin, g(h) with both exponential sums at the indices within 2 of it and
    at every 32nd index and the last, A = (4 pi)^(-1/2) S^(-1/2), and the
    PLUGIN values with the magnitude sums sum|K^(r)| of psi_6 at g1 and psi_4
    at g2 (the scales of their tolerances)."""
    from paper_1505_01998_gb300 import datagen
    n_h = 128
    sets = datagen.batch(512, seed=4)
    sizes = np.array([x.shape[1] for x in sets])
    above = sorted((int(n), i) for i, n in enumerate(sizes) if n > 16384)[:16]
    chosen = sorted([i for i, n in enumerate(sizes) if n <= 16384] + [i for _, i in above])
    cases = []
    for i in chosen:
        x = sets[i].astype(np.float64)  # the FP32 values the device sees
        n = x.shape[1]
        h = oracle.grid_default(n, 1, n_h)
        r = oracle.lscv_h(x, h)
        p = oracle.plugin(x[0])
        k0 = int(r["argmin"])
        idx = sorted(set(range(max(0, k0 - 2), min(n_h, k0 + 3))) | set(range(0, n_h, 32)) | {n_h - 1})
        _, S = oracle.mean_cov(x)
        case = {"i": i, "n": int(n), "argmin": k0, "idx": idx,
                "g": [float(r["g"][k]) for k in idx], "s_kk": [float(r["s_kk"][k]) for k in idx],
                "s_k": [float(r["s_k"][k]) for k in idx],
                "A": float((4 * np.pi) ** -0.5 / np.sqrt(S[0, 0])),
                "plugin_status": int(p["status"]),
                "plugin": {k: float(p[k]) for k in ("sigma", "g1", "psi6", "g2", "psi4", "h")}}
        if p["status"] == 0:
            case["psi6_abs"] = float(oracle.psi_abs_pair_sum(x[0], 6, p["g1"]))
            case["psi4_abs"] = float(oracle.psi_abs_pair_sum(x[0], 4, p["g2"]))
        cases.append(case)
        print(f"dataset {i}: n = {n}, argmin {k0}", flush=True)
    out = {
        "_about": "FP64 oracle of the 512-dataset batch (datagen.batch(512, seed=4)): every "
                  "dataset with n <= 16,384 and the 16 smallest above, LSCV_h on the 128-point "
                  "grid over Z(h0) (argmin; g and both exponential sums at sampled indices) and "
                  "the PLUGIN chain. Written by make_golden.py --batch; calls only the oracle.",
        "count": 512, "seed": 4, "n_h": n_h, "cases": cases,
    }
    with open(os.path.join(HERE, "batch512_oracle.json"), "w") as f:
        json.dump(out, f, separators=(",", ":"))


def main():
    if "--batch" in sys.argv:
        batch_subset()
        return
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
