"""Sharded LSCV_h on one GPU: the shards a multi-GPU run would give its ranks,
evaluated one after another and merged on the host, against the single
launch and the oracle."""
import numpy as np
import pytest

import oracle
from paper_1505_01998_gb300 import datagen
from paper_1505_01998_gb300.shard import tile_shards
from tests._helpers import TOL, built_lib, g_err, lscv_A

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("world", [2, 3, 8])
def test_sequential_shards_merge_to_the_single_launch(world):
    import torch
    kde = built_lib()
    n, d = 6000, 2
    x = datagen.correlated_mixture(n, d, seed=12)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    h = oracle.grid_default(n, d, 128)
    opts = kde.make_opts(tiles_per_item=4)
    tiles = kde.kde_tile_count(n, 128)
    s1 = np.zeros(h.size)
    s2 = np.zeros(h.size)
    for b, e in tile_shards(tiles, world, 4):
        a1, a2 = kde.kde_lscv_tile_sums(xd, h, b, e, opts)
        s1 += a1
        s2 += a2
    logdet = kde.kde_lscv_logdet(xd)
    res, g = kde.kde_lscv_merge(n, d, logdet, h, s1, s2)
    single, g1, _ = kde.kde_lscv(xd, kde.make_grid(h=h)[0], opts)
    assert np.allclose(g, g1, rtol=1e-12, atol=0)  # same items, FP64 merge order only
    assert res["argmin"] == single["argmin"]
    assert logdet == single["logdet_S"]
    x64 = x.astype(np.float32).astype(np.float64)
    ref = oracle.lscv_h(x64, h)
    err = g_err(g, ref["g"], ref["s_kk"], ref["s_k"], h, n, d, lscv_A(x64))
    assert err.max() < TOL


@pytest.mark.parametrize("world", [2, 3, 8])
def test_sequential_plugin_shards_match_the_single_call_and_oracle(world):
    """The psi_6 and psi_4 tile ranges a `world`-rank run would give its
    ranks, evaluated one after another on one GPU, summed on the host and
    advanced by kde_plugin_merge: equal to kde_plugin up to the FP64 order of
    the item sums (same items, default geometry), and to the oracle."""
    import torch

    from paper_1505_01998_gb300 import gbkde
    kde = built_lib()
    n = 20000
    x = datagen.skewed_column(n, seed=51)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    geo = gbkde.kde_item_tiles(n, 1, 0)
    shards = tile_shards(kde.kde_tile_count(n, geo["psi_tile"]), world, geo["psi_K"])
    sigma = float(np.sqrt(kde.kde_sample_covariance(xd)[0, 0]))
    res = kde.kde_plugin_merge(n, 8, sigma)
    for r, pilot in ((6, "g1"), (4, "g2")):
        total = sum(kde.kde_psi_tile_sums(xd, r, res[pilot], b, e) for b, e in shards)
        res = kde.kde_plugin_merge(n, r, total, res)
    single = kde.kde_plugin(xd)
    for k in ("g1", "psi6", "g2", "psi4", "h"):
        assert abs(res[k] - single[k]) <= 1e-11 * abs(single[k]), (k, res[k], single[k])
    ref = oracle.plugin(x.astype(np.float64)[0])
    for k in ("psi6", "psi4", "h"):
        assert abs(res[k] - ref[k]) <= TOL * abs(ref[k]), (k, res[k], ref[k])


def test_default_shards_fall_on_item_boundaries():
    """sharded_lscv with default options on one rank, and the shards of a
    4-rank run evaluated in turn with the default geometry's item size: the
    same items as the single launch."""
    import torch

    from paper_1505_01998_gb300 import gbkde
    from paper_1505_01998_gb300.shard import shard_item_tiles, sharded_lscv
    kde = built_lib()
    n, d = 9000, 1
    x = datagen.skewed_column(n, seed=52)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    h = oracle.grid_default(n, d, 64)
    single, g1, _ = kde.kde_lscv(xd, kde.make_grid(h=h)[0])
    res, g = sharded_lscv(xd, h)
    assert np.allclose(g, g1, rtol=1e-12, atol=0) and res["argmin"] == single["argmin"]
    geo = gbkde.kde_item_tiles(n, d, h.size, h=h)
    assert shard_item_tiles(n, d, h.size, h=h) == geo["lscv_K"]
    s1 = np.zeros(h.size)
    s2 = np.zeros(h.size)
    for b, e in tile_shards(kde.kde_tile_count(n, geo["lscv_tile"]), 4, geo["lscv_K"]):
        a1, a2 = kde.kde_lscv_tile_sums(xd, h, b, e)
        s1 += a1
        s2 += a2
    _, g4 = kde.kde_lscv_merge(n, d, kde.kde_lscv_logdet(xd), h, s1, s2)
    assert np.allclose(g4, g1, rtol=1e-12, atol=0)
