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
