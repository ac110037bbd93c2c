"""The LSCV geometry autotuner: the chosen geometry is valid, is used by later
calls that leave options at 0, and keeps results within tolerance."""
import numpy as np
import pytest

import oracle
from paper_1505_01998_gb300 import datagen
from tests._helpers import TOL, built_lib, g_err, lscv_A

pytestmark = pytest.mark.gpu


def test_autotune_picks_a_valid_geometry_and_later_calls_use_it(tmp_path):
    import torch
    kde = built_lib()
    kde.kde_autotune_clear()
    n, d, n_h = 12000, 1, 128
    x = datagen.skewed_column(n, seed=21)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    best, rate = kde.kde_autotune(xd, n_h, kde.KDE_TUNE_THROUGHPUT)
    assert best.tile in (32, 128) and best.bw_per_thread in (8, 16) and best.ctas_per_sm in (1, 2)
    assert best.tiles_per_item >= 1 and rate > 1e11
    h = oracle.grid_default(n, d, n_h)
    grid, keep = kde.make_grid(h=h)
    explicit = kde.make_opts(tile=best.tile, bw_per_thread=best.bw_per_thread,
                             tiles_per_item=best.tiles_per_item, ctas_per_sm=best.ctas_per_sm)
    r_auto, g_auto, _ = kde.kde_lscv(xd, grid)          # options at 0: the cached choice
    r_exp, g_exp, _ = kde.kde_lscv(xd, grid, explicit)  # the same geometry spelled out
    assert np.array_equal(g_auto, g_exp)
    x64 = x.astype(np.float32).astype(np.float64)
    ref = oracle.lscv_h(x64, h)
    assert g_err(g_auto, ref["g"], ref["s_kk"], ref["s_k"], h, n, d, lscv_A(x64)).max() < TOL
    path = tmp_path / "tune.txt"
    kde.kde_autotune_save(path)
    kde.kde_autotune_clear()
    kde.kde_autotune_load(path)
    r_again, g_again, _ = kde.kde_lscv(xd, grid)
    assert np.array_equal(g_again, g_auto)
    kde.kde_autotune_clear()
