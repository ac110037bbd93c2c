"""kde_lscv_noalloc: the LSCV_h entry point for callers that cannot allocate
device memory (an application allocator owning the device heap, code that
must not take cudaMalloc's implicit synchronisation, C callers without a
tensor library).  It uses a scratch buffer built into the library instead of
a caller workspace.  Collected last on purpose; runs alone or after the rest.
"""
import numpy as np
import pytest

import oracle
from paper_1505_01998_gb300 import datagen
from tests._helpers import TOL, built_lib

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))


def test_noalloc_matches_workspace_entry_point_on_consecutive_calls():
    kde = built_lib()
    cases = [(datagen.correlated_mixture(3000, 2, seed=31), 96),
             (datagen.skewed_column(20000, seed=32), 256)]
    for x, n_h in cases:  # two calls in a row share the built-in buffer
        d, n = x.shape
        h = oracle.grid_default(n, d, n_h)
        grid, keep = kde.make_grid(h=h)
        ref, g_ref, _ = kde.kde_lscv(_dev(x), grid)
        res, g, hh = kde.kde_lscv_noalloc(_dev(x), grid)
        assert res["status"] == 0
        assert np.array_equal(hh, h)
        assert _rel(g, g_ref) < TOL
        assert res["argmin"] == ref["argmin"]
        assert abs(res["h"] - ref["h"]) <= TOL * ref["h"]


def test_noalloc_rejects_problems_larger_than_its_buffer():
    kde = built_lib()
    x = _dev(np.zeros((4, 1 << 20), dtype=np.float32))
    grid, _ = kde.make_grid(n_h=256)
    with pytest.raises(kde.KdeError) as e:
        kde.kde_lscv_noalloc(x, grid)
    assert e.value.status == kde.KDE_ENOMEM
    assert "built-in" in str(e.value)
