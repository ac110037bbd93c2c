"""Host checks that the seeded generators draw the workloads as stated: the
n = 1,024 mixture (weights .5/.3/.2, means -2/0/3, sds .5/1/.8), the skewed
column (half lognormal(0, 1), half U[0, 100]), covariances with condition
number 50, batch sizes log-uniform on [256, 131072] and the serving mix
(Poisson arrivals, n log-uniform on [1024, 262144], d = 1 : 2 at 4 : 1,
LSCV : PLUGIN 1 : 1).  Moments are compared at several standard errors."""
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1505_01998_gb300 import datagen  # noqa: E402


def test_mixture_moments():
    x = datagen.mixture_1d(400000, seed=1)[0]
    w, mu, sd = np.array([0.5, 0.3, 0.2]), np.array([-2.0, 0.0, 3.0]), np.array([0.5, 1.0, 0.8])
    mean = float(w @ mu)
    var = float(w @ (sd ** 2 + mu ** 2)) - mean ** 2
    assert abs(x.mean() - mean) < 5 * math.sqrt(var / x.size)
    assert abs(x.var() - var) < 0.02 * var
    assert x.dtype == np.float64 and x.shape == (400000,)


def test_skewed_column_halves():
    x = datagen.skewed_column(65536, seed=2)
    assert x.shape == (1, 65536) and x.dtype == np.float32
    v = x[0].astype(np.float64)
    assert v.min() >= 0.0
    n = v.size
    # below 1: half the lognormal part, 1 % of the uniform part
    p_lt1 = 0.5 * 0.5 + 0.5 * 0.01
    assert abs((v < 1.0).mean() - p_lt1) < 5 * math.sqrt(p_lt1 * (1 - p_lt1) / n)
    # above 30: 70 % of the uniform part (the lognormal tail is 3.4e-4)
    p_gt30 = 0.5 * 0.7 + 0.5 * 0.5 * math.erfc(math.log(30.0) / math.sqrt(2.0))
    assert abs((v > 30.0).mean() - p_gt30) < 5 * math.sqrt(p_gt30 * (1 - p_gt30) / n)
    # above 100 only the lognormal tail (2e-6 per draw)
    assert (v > 100.0).sum() <= 3


def test_covariances_have_condition_number_50():
    g = datagen.rng(9)
    for d in (1, 2, 3, 4, 8, 16):
        S = datagen.random_spd(d, g)
        assert np.allclose(S, S.T, atol=1e-12)
        lam = np.linalg.eigvalsh(S)
        assert abs(lam[0] - 1.0) < 1e-9
        if d >= 2:
            assert abs(lam[-1] - 50.0) < 1e-9
        assert lam.min() > 0


def test_batch_sizes_log_uniform():
    s = datagen.batch_sizes(512, 4)
    assert s.min() >= 256 and s.max() <= 131072
    lg = np.log2(s.astype(np.float64))
    # log2 n uniform on [8, 17]: mean 12.5, sd 9 / sqrt(12)
    assert abs(lg.mean() - 12.5) < 5 * (9 / math.sqrt(12)) / math.sqrt(s.size)


def test_serving_mix():
    reqs = datagen.serving_requests(100.0, 6000, seed=5, materialise=False)
    n = np.array([r.n for r in reqs], dtype=np.float64)
    assert n.min() >= 1024 and n.max() <= 262144
    d2 = np.mean([r.d == 2 for r in reqs])
    assert abs(d2 - 0.2) < 5 * math.sqrt(0.2 * 0.8 / len(reqs))
    plug = np.mean([r.method == "plugin" for r in reqs])
    assert abs(plug - 0.5) < 5 * math.sqrt(0.25 / len(reqs))
    assert all(r.method == "lscv" for r in reqs if r.d == 2)
    gaps = np.diff([0.0] + [r.arrival_s for r in reqs])
    assert gaps.min() > 0
    assert abs(gaps.mean() - 0.01) < 5 * 0.01 / math.sqrt(len(reqs))
