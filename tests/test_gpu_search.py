"""Exact leave-one-out weights and the bracketing search, against the oracle."""
import numpy as np
import pytest

import oracle
from paper_1505_01998_gb300 import datagen
from tests._helpers import TOL, built_lib, g_err, lscv_A

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


@pytest.mark.parametrize("d,n", [(1, 1500), (2, 900), (3, 2500)])
def test_loo_objective_matches_oracle(d, n):
    kde = built_lib()
    x = datagen.correlated_mixture(n, d, seed=70 + d)
    x64 = x.astype(np.float32).astype(np.float64)
    h = oracle.grid_default(n, d, 64)
    res, g, _ = kde.kde_lscv(_dev(x), kde.make_grid(h=h)[0], kde.make_opts(cv=kde.KDE_CV_LOO))
    ref = oracle.lscv_h_loo(x64, h)
    s = oracle.lscv_sums(x64, h)
    err = g_err(g, ref, s[0], s[1], h, n, d, lscv_A(x64))
    assert err.max() < TOL
    assert res["argmin"] == int(np.argmin(ref)) or ref[res["argmin"]] - ref.min() <= TOL * np.abs(ref).max()


@pytest.mark.parametrize("d,n,loo", [(1, 3000, False), (1, 800, True), (2, 2000, False)])
def test_search_matches_oracle_search(d, n, loo):
    kde = built_lib()
    x = datagen.correlated_mixture(n, d, seed=90 + d + n)
    x64 = x.astype(np.float32).astype(np.float64)
    z = oracle.h0(n, d)
    opts = kde.make_opts(cv=kde.KDE_CV_LOO if loo else kde.KDE_CV_PAPER)
    res, rounds = kde.kde_lscv_search(_dev(x), z / 4, 4 * z, rel_tol=1e-3, opts=opts)
    hs, gs, rounds_o = oracle.lscv_search(x64, z / 4, 4 * z, P=8, rel_tol=1e-3, loo=loo)
    assert rounds == rounds_o
    # the same bracket decisions give the same point; a near tie may pick a neighbour
    assert abs(np.log(res["h"] / hs)) <= np.log(4 * z / (z / 4)) * (2 / 9) ** (rounds - 1)
    g_at = (oracle.lscv_h_loo(x64, [res["h"]])[0] if loo else oracle.lscv_h(x64, [res["h"]])["g"][0])
    assert abs(g_at - gs) <= 1e-5 * abs(gs)
    assert abs(res["g_min"] - g_at) <= 1e-5 * abs(g_at)


def test_search_is_no_worse_than_the_dense_grid():
    """Interior minimum (three-component mixture): the search ends at or below
    the best point of a 256-point grid over the same range, without edge flags."""
    kde = built_lib()
    n = 20000
    x = datagen.mixture_1d(n, seed=17)
    res, rounds = kde.kde_lscv_search(_dev(x), rel_tol=1e-4)
    grid_res, g, h = kde.kde_lscv(_dev(x), kde.make_grid(n_h=256)[0])
    assert 0 < grid_res["argmin"] < 255
    assert res["g_min"] <= grid_res["g_min"] + 1e-6 * abs(grid_res["g_min"])
    assert res["flags"] == 0
    assert rounds <= 10


def test_search_flags_a_minimum_at_the_range_end():
    """The skewed column's g(h) still falls at h0/4 (the dense grid's argmin is
    its first point): the search walks down to the lower end and flags it."""
    kde = built_lib()
    n = 20000
    x = datagen.skewed_column(n, seed=17)
    res, rounds = kde.kde_lscv_search(_dev(x), rel_tol=1e-4)
    grid_res, g, h = kde.kde_lscv(_dev(x), kde.make_grid(n_h=256)[0])
    assert grid_res["argmin"] == 0
    assert res["flags"] == kde.KDE_FLAG_MIN_AT_LOWER_EDGE
    assert abs(np.log(res["h"] / h[0])) <= 2e-4
