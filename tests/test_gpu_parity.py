"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Inputs are the same FP32 values on both sides (the oracle widens them to
FP64), except where an FP64 input path is under test.  Tolerances and error
metrics: see tests/_helpers.py.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1505_01998_gb300 import datagen
from tests._helpers import TOL, argmin_ok, built_lib, g_err, lscv_A, rel_err, s_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kde():
    return built_lib()


def dev(x, dtype="float32"):
    import torch
    a = np.ascontiguousarray(np.asarray(x))
    if a.ndim == 1:
        a = a[None, :]
    return torch.from_numpy(a.astype(dtype)).cuda()


def host64(x, dtype="float32"):
    a = np.asarray(x)
    if a.ndim == 1:
        a = a[None, :]
    return a.astype(dtype).astype(np.float64)


def oracle_tile_sums_lscv(x64, h, T, tb, te, kde):
    s1 = np.zeros(len(h))
    s2 = np.zeros(len(h))
    for t in range(tb, te):
        l, q = kde.kde_tile_coords(t)
        a, b, _ = oracle.lscv_sums(x64, h, block=(q * T, q * T + T, l * T, l * T + T))
        s1 += a
        s2 += b
    return s1, s2


def oracle_tile_sums_psi(x64, r, g, T, tb, te, kde):
    s = 0.0
    sa = 0.0
    for t in range(tb, te):
        l, q = kde.kde_tile_coords(t)
        blk = (q * T, q * T + T, l * T, l * T + T)
        s += oracle.psi_pair_sum(x64, r, g, block=blk)
        sa += oracle.psi_abs_pair_sum(x64, r, g, block=blk)
    return s, sa


# ----------------------------------------------------------------- psi

@pytest.mark.parametrize("n", [2, 3, 65, 1000, 20000])
@pytest.mark.parametrize("r", [4, 6, 8])
def test_psi_full_range_sums(kde, n, r):
    x = datagen.mixture_1d(n, seed=10 + n)[0]
    xd = dev(x)
    x64 = host64(x)[0]
    T = kde.kde_psi_tile_edge(n)
    tiles = kde.kde_tile_count(n, T)
    for g in (0.05, 0.4, 2.0):
        got = kde.kde_psi_tile_sums(xd, r, g, 0, tiles)
        ref = oracle.psi_pair_sum(x64, r, g)
        mag = oracle.psi_abs_pair_sum(x64, r, g)
        assert abs(got - ref) <= TOL * max(abs(ref), mag) + 1e-300, (g, got, ref, mag)


@pytest.mark.parametrize("n", [300, 5000])
def test_psi_tile_ranges_add_up(kde, n):
    x = datagen.skewed_column(n, seed=3)[0]
    xd = dev(x)
    x64 = host64(x)[0]
    T = kde.kde_psi_tile_edge(n)
    tiles = kde.kde_tile_count(n, T)
    cuts = [0, 1, tiles // 3, tiles - 1, tiles]
    parts = [kde.kde_psi_tile_sums(xd, 6, 3.0, cuts[k], cuts[k + 1]) for k in range(4)]
    full = kde.kde_psi_tile_sums(xd, 6, 3.0, 0, tiles)
    # different tile ranges group tiles into different items (different FP32
    # runs), so the split agrees with the whole to FP32 rounding of the terms
    mag_all = oracle.psi_abs_pair_sum(x64, 6, 3.0)
    assert abs(sum(parts) - full) <= 1e-6 * mag_all
    assert abs(full - oracle.psi_pair_sum(x64, 6, 3.0)) <= TOL * mag_all
    ref, mag = oracle_tile_sums_psi(x64, 6, 3.0, T, cuts[3], cuts[4], kde)
    assert abs(parts[3] - ref) <= TOL * max(abs(ref), mag)


def test_psi_largest_tiles_ragged_tail(kde):
    """n = 65,869 (a ragged last tile column): psi tiles of 512 (two row
    groups of 256 rows per CTA) against the oracle's block sums on the first
    tiles (two diagonal), a middle range and the ragged last column, and the
    full range of psi_6 against the oracle's whole double sum."""
    n = 65536 + 333
    x = datagen.skewed_column(n, seed=41)[0]
    xd = dev(x)
    x64 = host64(x)[0]
    T = kde.kde_psi_tile_edge(n)
    assert T == 512
    tiles = kde.kde_tile_count(n, T)
    for r, g in ((6, 3.0), (4, 0.7)):
        for tb, te in ((0, 3), (tiles // 2, tiles // 2 + 2), (tiles - 3, tiles)):
            got = kde.kde_psi_tile_sums(xd, r, g, tb, te)
            ref, mag = oracle_tile_sums_psi(x64, r, g, T, tb, te, kde)
            assert abs(got - ref) <= TOL * max(abs(ref), mag), (r, tb, te, got, ref, mag)
    got = kde.kde_psi_tile_sums(xd, 6, 3.0, 0, tiles)
    ref = oracle.psi_pair_sum(x64, 6, 3.0)
    mag = oracle.psi_abs_pair_sum(x64, 6, 3.0)
    assert abs(got - ref) <= TOL * max(abs(ref), mag), (got, ref, mag)


# -------------------------------------------------------------- plug-in

def _plugin_compare(res, ref, x64):
    assert res["status"] == ref["status"] == 0
    assert rel_err(res["sigma"], ref["sigma"]) < 1e-6
    assert rel_err(res["g1"], ref["g1"]) < 1e-6
    n = x64.size
    for key, r, gk in (("psi6", 6, "g1"), ("psi4", 4, "g2")):
        g = ref[gk]
        mag = (2 * oracle.psi_abs_pair_sum(x64, r, g) + n * abs(oracle.gauss_deriv(r, 0.0))) / (
            n * n * g ** (r + 1))
        assert abs(res[key] - ref[key]) <= TOL * max(abs(ref[key]), mag), (key, res[key], ref[key])
    assert rel_err(res["g2"], ref["g2"]) < TOL
    assert rel_err(res["h"], ref["h"]) < TOL
    assert res["h_data"] == res["h"]


@pytest.mark.parametrize("n,dtype", [(1024, "float64"), (777, "float32"), (5000, "float32"),
                                     (20000, "float32")])
def test_plugin_matches_oracle(kde, n, dtype):
    x = datagen.mixture_1d(n, seed=1)[0] if n == 1024 else datagen.skewed_column(n, seed=n)[0]
    res = kde.kde_plugin(dev(x, dtype))
    x64 = host64(x, dtype)[0]
    _plugin_compare(res, oracle.plugin(x64), x64)


@pytest.mark.parametrize("n,seed", [(1024, 1), (3000, 7), (65536, 2)])
def test_plugin_chain_roots_match_library_roots(kde, n, seed):
    """The device forms g2 = (-2 K4(0) / (psi6 n))^(1/7) and
    h = (R(K) / (psi4 n))^(1/5) by Newton's iteration for the inverse root
    from an FP32 seed, and sigma from one reciprocal square root: each agrees
    with numpy's FP64 power of the device's own chain values (psi6, psi4 and
    the sample variance, in the kernel's FP32 samples) to a few units in the
    last place.  The arguments differ from numpy's by the order of their
    divisions (at most a few ulp), which the root divides by 7 or 5; sigma is
    checked against the device's own log|S|."""
    x = datagen.mixture_1d(n, seed=seed)[0] if n < 65536 else datagen.skewed_column(n, seed=seed)[0]
    res = kde.kde_plugin(dev(x))
    k4_0 = 3.0 / math.sqrt(2.0 * math.pi)
    rk = 1.0 / (2.0 * math.sqrt(math.pi))
    g2 = np.power(-2.0 * k4_0 / (res["psi6"] * n), 1.0 / 7.0)
    h = np.power(rk / (res["psi4"] * n), 0.2)
    assert abs(res["g2"] - g2) <= 4e-15 * g2, (res["g2"], g2)
    assert abs(res["h"] - h) <= 4e-15 * h, (res["h"], h)
    # sigma = sqrt(S_00), S_00 = exp(log|S|) for d = 1; g1 = sigma c_g1
    sigma = math.sqrt(math.exp(res["logdet_S"]))
    assert abs(res["sigma"] - sigma) <= 1e-14 * sigma, (res["sigma"], sigma)
    c_g1 = np.power(2.0 * 15.0 / math.sqrt(2.0 * math.pi) * 32.0 * math.sqrt(math.pi) / (105.0 * n), 1.0 / 9.0)
    assert abs(res["g1"] - res["sigma"] * c_g1) <= 4e-15 * res["g1"], (res["g1"], res["sigma"] * c_g1)


def test_plugin_plain_precision_also_within_tolerance(kde):
    x = datagen.mixture_1d(3000, seed=4)[0]
    x64 = host64(x)[0]
    res = kde.kde_plugin(dev(x), kde.make_opts(precision=kde.KDE_FP32_PLAIN))
    _plugin_compare(res, oracle.plugin(x64), x64)


# ------------------------------------------------------------------ LSCV

def _lscv_check(kde, x, h, opts=None, dtype="float32"):
    xd = dev(x, dtype)
    x64 = host64(x, dtype)
    d, n = x64.shape
    res, g, hh = kde.kde_lscv(xd, _explicit(kde, h), opts)
    assert np.array_equal(hh, np.asarray(h, dtype=np.float64))
    ref = oracle.lscv_h(x64, h)
    A = lscv_A(x64)
    err = g_err(g, ref["g"], ref["s_kk"], ref["s_k"], h, n, d, A)
    assert err.max() < TOL, (err.max(), int(err.argmax()))
    # exponential sums over the whole triangle
    T = kde.kde_item_tiles(n, d, len(h), opts, h=h)["lscv_tile"]
    tiles = kde.kde_tile_count(n, T)
    s1, s2 = kde.kde_lscv_tile_sums(xd, h, 0, tiles, opts)
    npairs = n * (n - 1) // 2
    assert s_err(s1, ref["s_kk"], npairs).max() < TOL
    assert s_err(s2, ref["s_k"], npairs).max() < TOL
    assert argmin_ok(res["argmin"], ref["g"], TOL * np.max(np.abs(ref["g"])))
    assert res["n_h"] == len(h) and res["d"] == d
    assert res["h"] == h[res["argmin"]]
    if d == 1:
        assert rel_err(res["h_data"], h[res["argmin"]] * math.sqrt(np.var(x64, ddof=1))) < 1e-6
    return res, g, ref


_keep = []


def _explicit(kde, h):
    grid, arr = kde.make_grid(h=h)
    _keep.append(arr)
    return grid


def test_lscv_n1024_mixture_64_point_grid(kde):
    """The n = 1,024 FP64 mixture with a 64-point log grid over [0.01, 2]."""
    x = datagen.mixture_1d(1024, seed=1)
    h = oracle.grid_log(0.01, 2.0, 64)
    _lscv_check(kde, x, h, dtype="float64")
    _lscv_check(kde, x, h, dtype="float32")


@pytest.mark.parametrize("d", [1, 2, 3, 4])
@pytest.mark.parametrize("n,n_h", [(700, 64), (2100, 128), (333, 12), (1500, 40), (2500, 256)])
def test_lscv_dims_sizes_grids(kde, d, n, n_h):
    x = datagen.correlated_mixture(n, d, seed=7 * d + n)
    h = oracle.grid_default(n, d, n_h)
    _lscv_check(kde, x, h)


@pytest.mark.parametrize("d", [1, 3, 6, 16])
@pytest.mark.parametrize("n,n_h", [(1100, 1), (2000, 2), (3001, 1), (5000, 2)])
def test_lscv_one_and_two_point_grids(kde, d, n, n_h):
    """Grids of one or two points take 2 bandwidths per thread (one g(H) of
    LSCV_H is such a grid); d = 6 and 16 also prefetch the next tile's rows;
    above n = 2,048 d <= 4 takes tiles of 256 (8 rows per lane) and a
    one-point grid pairs rows in the packed evaluation."""
    x = datagen.correlated_mixture(n, d, seed=500 + d + n)
    h = oracle.grid_default(n, d, 8)[3:3 + n_h]
    _lscv_check(kde, x, h)


@pytest.mark.parametrize("d", [5, 7, 8, 9, 12, 13, 16])
@pytest.mark.parametrize("n,n_h", [(450, 32), (1300, 100)])
def test_lscv_high_dimensions(kde, d, n, n_h):
    """d = 5..16 (the paper's experiments reach d = 16): coordinates padded to
    8 / 12 / 16 with zeros, one row per lane."""
    x = datagen.correlated_mixture(n, d, seed=300 + d + n)
    h = oracle.grid_default(n, d, n_h)
    _lscv_check(kde, x, h)


@pytest.mark.parametrize("d", [6, 16])
def test_lscv_H_high_dimensions(kde, d):
    n = 700
    x = datagen.correlated_mixture(n, d, seed=400 + d)
    x64 = x.astype(np.float32).astype(np.float64)
    _, S = oracle.mean_cov(x64)
    Hs = np.array([0.3 * S, 0.8 * S + 0.1 * np.eye(d)])
    g = kde.kde_lscv_H(dev(x), Hs)
    for k in range(2):
        ref = oracle.lscv_H(x64, Hs[k])
        scale = (4 * math.pi) ** (-d / 2) / math.sqrt(np.linalg.det(Hs[k])) / n
        assert abs(g[k] - ref) <= TOL * max(abs(ref), scale)


@pytest.mark.parametrize("opts", [dict(precision=1), dict(tile=128), dict(tile=32, bw_per_thread=16),
                                  dict(bw_per_thread=8, tiles_per_item=3), dict(ctas_per_sm=1),
                                  dict(bw_per_thread=2), dict(tile=32, bw_per_thread=2, precision=1)])
def test_lscv_option_paths(kde, opts):
    x = datagen.correlated_mixture(1800, 2, seed=99)
    h = oracle.grid_default(1800, 2, 96)
    _lscv_check(kde, x, h, kde.make_opts(**opts))


def test_lscv_deterministic_and_grid_independent(kde):
    x = datagen.skewed_column(5000, seed=12)
    xd = dev(x)
    grid = _explicit(kde, oracle.grid_default(5000, 1, 128))
    # item partials depend only on the tile partition (K), not on the grid size
    r1, g1, _ = kde.kde_lscv(xd, grid, kde.make_opts(tiles_per_item=5))
    r2, g2, _ = kde.kde_lscv(xd, grid, kde.make_opts(tiles_per_item=5))
    r3, g3, _ = kde.kde_lscv(xd, grid, kde.make_opts(tiles_per_item=5, ctas_per_sm=1))
    assert np.array_equal(g1, g2) and np.array_equal(g1, g3)
    assert r1 == r2 == r3


def test_lscv_tile_ranges_add_up(kde):
    x = datagen.correlated_mixture(3000, 3, seed=5)
    xd = dev(x)
    h = oracle.grid_default(3000, 3, 64)
    tiles = kde.kde_tile_count(3000, 128)
    cuts = [0, 5, tiles // 2, tiles - 2, tiles]
    s1 = np.zeros(64)
    s2 = np.zeros(64)
    for k in range(4):
        a, b = kde.kde_lscv_tile_sums(xd, h, cuts[k], cuts[k + 1])
        s1 += a
        s2 += b
    f1, f2 = kde.kde_lscv_tile_sums(xd, h, 0, tiles)
    # positive terms; regrouped FP32 runs agree to FP32 rounding
    assert np.allclose(s1, f1, rtol=1e-6) and np.allclose(s2, f2, rtol=1e-6)


def test_lscv_host_and_async_paths_match(kde):
    import torch
    x = datagen.correlated_mixture(2500, 2, seed=8)
    grid = _explicit(kde, oracle.grid_default(2500, 2, 128))
    r1, g1, _ = kde.kde_lscv(dev(x), grid)
    ws = kde.workspace(kde.kde_workspace_size(2500, 2, 128))
    r2, g2 = kde.kde_lscv_host(np.ascontiguousarray(x, dtype=np.float32), grid, None, ws)
    assert np.array_equal(g1, g2) and r1 == r2
    kde.kde_lscv_async(dev(x), grid, None, ws)
    torch.cuda.synchronize()
    r3, g3 = kde.read_ws_result(ws, 128)
    assert np.array_equal(g1, g3) and r3 == r1


def test_back_to_back_async_calls_on_one_stream(kde):
    """Single calls launch with programmatic dependent launch: each kernel
    may be scheduled while the previous one drains and waits (PTX
    griddepcontrol.wait) before touching memory.  Queued without any
    synchronisation on one stream -- samples written by a torch kernel just
    before, a workspace reused while the earlier selection that used it may
    still run, LSCV and PLUGIN interleaved -- every result equals the same
    call made alone and synchronised."""
    import torch
    n1, n2, n3 = 3000, 1000, 20000
    xa = datagen.mixture_1d(n1, seed=31)[0].astype(np.float32)
    xb = datagen.skewed_column(n2, seed=32)[0].astype(np.float32)
    xc = datagen.skewed_column(n3, seed=33)[0].astype(np.float32)
    ga = _explicit(kde, oracle.grid_log(0.02, 2.0, 64))
    gc = _explicit(kde, oracle.grid_default(n3, 1, 256))
    ref_a = kde.kde_lscv(dev(xa), ga)
    ref_b = kde.kde_plugin(dev(xb))
    ref_c = kde.kde_lscv(dev(xc), gc)
    ws1 = kde.workspace(max(kde.kde_workspace_size(n, 1, 256) for n in (n1, n3)))
    ws2 = kde.workspace(kde.kde_workspace_size(n2, 1, 0))
    da, db, dc = (torch.empty((1, n), dtype=torch.float32, device="cuda") for n in (n1, n2, n3))
    src = [dev(x) for x in (xa, xb, xc)]
    torch.cuda.synchronize()
    for rep in range(3):
        for t, sx in zip((da, db, dc), src):
            t.fill_(float("nan"))
            torch.add(sx, 0.0, out=t)  # the samples come from a torch kernel right before the calls
        kde.kde_lscv_async(da, ga, None, ws1)
        kde.kde_plugin_async(db, None, ws2)
        torch.cuda.synchronize()
        res_a, g_a = kde.read_ws_result(ws1, 64)
        assert res_a == ref_a[0] and np.array_equal(g_a, ref_a[1]), rep
        kde.kde_lscv_async(da, ga, None, ws1)
        kde.kde_plugin_async(db, None, ws2)
        kde.kde_lscv_async(dc, gc, None, ws1)  # ws1 reused right behind the first selection
        torch.cuda.synchronize()
        res_c, g_c = kde.read_ws_result(ws1, 256)
        res_b, _ = kde.read_ws_result(ws2, 0)
        assert res_c == ref_c[0] and np.array_equal(g_c, ref_c[1]), rep
        assert res_b == ref_b, rep


def test_single_calls_captured_in_a_cuda_graph(kde):
    """Async single calls captured into a CUDA graph by the caller (their
    programmatic dependent launches become graph edges) and replayed: the
    results equal those of the same calls made directly, on every replay."""
    import torch
    n = 5000
    x = datagen.skewed_column(n, seed=41)[0].astype(np.float32)
    grid = _explicit(kde, oracle.grid_default(n, 1, 128))
    ref_l = kde.kde_lscv(dev(x), grid)
    ref_p = kde.kde_plugin(dev(x))
    xd = dev(x)
    ws_l = kde.workspace(kde.kde_workspace_size(n, 1, 128))
    ws_p = kde.workspace(kde.kde_workspace_size(n, 1, 0))
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        st = torch.cuda.current_stream()
        kde.kde_lscv_async(xd, grid, None, ws_l, st)
        kde.kde_plugin_async(xd, None, ws_p, st)
    for _ in range(3):
        ws_l.zero_()
        ws_p.zero_()
        graph.replay()
        torch.cuda.synchronize()
        res_l, g_l = kde.read_ws_result(ws_l, 128)
        res_p, _ = kde.read_ws_result(ws_p, 0)
        assert res_l == ref_l[0] and np.array_equal(g_l, ref_l[1])
        assert res_p == ref_p


# ------------------------------------------------------------ edge cases

def test_two_and_three_samples(kde):
    for x in (np.array([[0.3, 1.7]]), np.array([[0.0, 0.5, 2.0]])):
        h = np.array([0.2, 0.7, 1.5])
        _lscv_check(kde, x, h)
        ref = oracle.plugin(host64(x)[0])
        if ref["status"] == 0:
            _plugin_compare(kde.kde_plugin(dev(x)), ref, host64(x)[0])
        else:
            with pytest.raises(kde.KdeError) as e:
                kde.kde_plugin(dev(x))
            assert e.value.status == kde.KDE_EDEGENERATE


@pytest.mark.parametrize("n", [32, 33, 64, 2048, 2049])
def test_tile_boundaries(kde, n):
    x = datagen.mixture_1d(n, seed=n)
    _lscv_check(kde, x, oracle.grid_default(n, 1, 16))


def test_degenerate_inputs_reported(kde):
    const = np.full((1, 100), 3.0)
    with pytest.raises(kde.KdeError) as e:
        kde.kde_lscv(dev(const), _explicit(kde, [0.5, 1.0]))
    assert e.value.status == kde.KDE_EDEGENERATE
    with pytest.raises(kde.KdeError) as e:
        kde.kde_plugin(dev(const))
    assert e.value.status == kde.KDE_EDEGENERATE
    t = np.linspace(0, 1, 50)
    collinear = np.stack([t, 2 * t + 1])
    with pytest.raises(kde.KdeError) as e:
        kde.kde_lscv(dev(collinear), _explicit(kde, [0.5, 1.0]))
    assert e.value.status == kde.KDE_EDEGENERATE
    bad = datagen.mixture_1d(100, seed=1)
    bad[0, 7] = np.nan
    with pytest.raises(kde.KdeError) as e:
        kde.kde_lscv(dev(bad), _explicit(kde, [0.5, 1.0]))
    assert e.value.status == kde.KDE_EINVAL
    # the library stays usable after device-reported errors
    _lscv_check(kde, datagen.mixture_1d(200, seed=2), np.array([0.3, 0.6]))


def test_workspace_too_small_is_reported(kde):
    x = datagen.mixture_1d(5000, seed=3)
    need = kde.kde_workspace_size(5000, 1, 64)
    ws = kde.workspace(need - 1024)
    with pytest.raises(kde.KdeError) as e:
        kde.kde_lscv(dev(x), _explicit(kde, oracle.grid_default(5000, 1, 64)), None, ws)
    assert e.value.status == kde.KDE_ENOMEM


# ------------------------------------------- full-size workloads (sampled)

def test_full_size_skewed_column_sampled_tiles(kde):
    """n = 65,536 skewed column, 256-point grid over Z(h0), the launch
    configuration of the benchmark: sampled tiles against the oracle, tile-range
    additivity, plug-in chain consistency."""
    n = 65536
    x = datagen.skewed_column(n, seed=2)
    xd = dev(x)
    x64 = host64(x)
    h = oracle.grid_default(n, 1, 256)
    res, g, _ = kde.kde_lscv(xd, _explicit(kde, h))
    assert res["status"] == 0 and np.all(np.isfinite(g))
    T = 128
    tiles = kde.kde_tile_count(n, T)
    for tb, te in ((0, 3), (tiles // 2, tiles // 2 + 2), (tiles - 3, tiles)):
        s1, s2 = kde.kde_lscv_tile_sums(xd, h, tb, te)
        r1, r2 = oracle_tile_sums_lscv(x64, h, T, tb, te, kde)
        assert s_err(s1, r1, (te - tb) * T * T).max() < TOL
        assert s_err(s2, r2, (te - tb) * T * T).max() < TOL
    # plug-in: sigma/g1 against the oracle, psi tile samples at the device's pilots
    p = kde.kde_plugin(xd)
    m, S = oracle.mean_cov(x64)
    sig = math.sqrt(S[0, 0])
    assert rel_err(p["sigma"], sig) < 1e-6
    assert rel_err(p["g1"], oracle.plugin_g1(oracle.psi8_ns(sig), n)) < 1e-6
    Tp = kde.kde_psi_tile_edge(n)
    ptiles = kde.kde_tile_count(n, Tp)
    for r, gp in ((6, p["g1"]), (4, p["g2"])):
        for tb, te in ((0, 2), (ptiles - 2, ptiles)):
            got = kde.kde_psi_tile_sums(xd, r, gp, tb, te)
            ref, mag = oracle_tile_sums_psi(x64[0], r, gp, Tp, tb, te, kde)
            assert abs(got - ref) <= TOL * max(abs(ref), mag)
        full = kde.kde_psi_tile_sums(xd, r, gp, 0, ptiles)
        psi = (2 * full + n * oracle.gauss_deriv(r, 0.0)) / (n * n * gp ** (r + 1))
        assert psi == pytest.approx(p["psi6" if r == 6 else "psi4"], rel=1e-12)
    assert rel_err(p["g2"], oracle.plugin_g2(p["psi6"], n)) < 1e-12
    assert rel_err(p["h"], oracle.plugin_h(p["psi4"], n)) < 1e-12


def test_full_size_skewed_column_against_full_oracle(kde):
    """The benchmark selection (n = 65,536 skewed column, 256-point grid over
    Z(h0), default launch geometry, Kahan FP32) against the FP64 oracle over
    all 2.1e9 pairs, stored by tests/golden/make_golden.py --full-skewed:
    S1, S2 and g(h) at every grid point, the argmin, and the PLUGIN chain."""
    import json
    import os
    ref = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "skewed65536_oracle.json")))
    n = ref["n"]
    x = datagen.skewed_column(n, seed=ref["seed"])
    xd = dev(x)
    x64 = host64(x)
    h = np.asarray(ref["h"])
    grid, _ = kde.make_grid(n_h=256)
    res, g, hh = kde.kde_lscv(xd, grid)
    assert np.allclose(hh, h, rtol=1e-15, atol=0)
    s_kk, s_k, g_ref = np.asarray(ref["s_kk"]), np.asarray(ref["s_k"]), np.asarray(ref["g"])
    err = g_err(g, g_ref, s_kk, s_k, h, n, 1, lscv_A(x64))
    assert err.max() < TOL, (err.max(), int(err.argmax()))
    assert argmin_ok(res["argmin"], g_ref, TOL * np.max(np.abs(g_ref)))
    tiles = kde.kde_tile_count(n, 128)
    s1, s2 = kde.kde_lscv_tile_sums(xd, h, 0, tiles)
    npairs = n * (n - 1) // 2
    assert s_err(s1, s_kk, npairs).max() < TOL
    assert s_err(s2, s_k, npairs).max() < TOL
    p = kde.kde_plugin(xd)
    rp = ref["plugin"]
    for key in ("sigma", "g1", "psi6", "g2", "psi4"):
        assert rel_err(p[key], rp[key]) < TOL, (key, p[key], rp[key])
    assert rel_err(p["h"], rp["h"]) < TOL


@pytest.mark.parametrize("d", [2, 3, 4])
def test_full_size_correlated_mixture(kde, d):
    """n = 16,384, d = 2..4, H = h^2 S on the 128-point default grid, default
    launch geometry, Kahan FP32, against the FP64 oracle over all 1.3e8 pairs
    stored by tests/golden/make_golden.py --full-mixture: g(h), S1 and S2 at
    every grid point and the argmin."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "mixture16384_oracle.json")))
    ref = gold["cases"][str(d)]
    n = gold["n"]
    x = datagen.correlated_mixture(n, d, seed=ref["seed"])
    xd = dev(x)
    x64 = host64(x)
    h = np.asarray(ref["h"])
    res, g, hh = kde.kde_lscv(xd, kde.make_grid(n_h=gold["n_h"])[0])
    assert np.allclose(hh, h, rtol=1e-15, atol=0)
    s_kk, s_k, g_ref = np.asarray(ref["s_kk"]), np.asarray(ref["s_k"]), np.asarray(ref["g"])
    err = g_err(g, g_ref, s_kk, s_k, h, n, d, lscv_A(x64))
    assert err.max() < TOL, (err.max(), int(err.argmax()))
    assert argmin_ok(res["argmin"], g_ref, TOL * np.max(np.abs(g_ref)))
    T = 128
    tiles = kde.kde_tile_count(n, T)
    s1, s2 = kde.kde_lscv_tile_sums(xd, h, 0, tiles)
    npairs = n * (n - 1) // 2
    assert s_err(s1, s_kk, npairs).max() < TOL
    assert s_err(s2, s_k, npairs).max() < TOL


@pytest.mark.parametrize("n,d,dtype", [(1025, 1, "float32"), (131073, 3, "float32"), (300001, 2, "float64"),
                                       (70001, 16, "float32"), (5000, 12, "float64")])
def test_prologue_statistics_across_ranges(kde, n, d, dtype):
    """The prologue cuts the samples into up to 128 ranges and combines their
    moments: sample covariance and log|S| against the oracle for sizes that
    give 2 and 128 ranges with ragged ends, FP32 and FP64 input.  The mean
    is offset far from zero so that centring errors would show."""
    x = datagen.correlated_mixture(n, d, seed=500 + d) if d > 1 else datagen.mixture_1d(n, seed=501)
    x = (np.asarray(x, dtype=np.float64) + 40.0).astype(dtype)
    x64 = host64(x, dtype)
    xd = dev(x, dtype)
    _, S_ref = oracle.mean_cov(x64)
    S = kde.kde_sample_covariance(xd)
    scale = np.sqrt(np.outer(np.diag(S_ref), np.diag(S_ref)))
    assert (np.abs(S - S_ref) / scale).max() < 1e-6
    logdet = kde.kde_lscv_logdet(xd)
    assert abs(logdet - np.linalg.slogdet(S_ref)[1]) < 1e-5 * max(1.0, abs(np.linalg.slogdet(S_ref)[1])) * d


def test_octave_kernel_input_types_precisions_and_grid_shapes(kde):
    """The octave kernel with FP64 samples, with plain FP32 sums, with the
    smallest octave grid (16 points, 2 per octave), and a grid of that shape
    given explicitly (bitwise the default grid's result).  A grid one part in
    1e9 off the octave shape takes the direct kernel, also within tolerance."""
    x = datagen.mixture_1d(4000, seed=611)
    h = oracle.grid_default(4000, 1, 128)
    _lscv_check(kde, x, h, dtype="float64")
    _lscv_check(kde, x, h, opts=kde.make_opts(precision=kde.KDE_FP32_PLAIN))
    x3 = datagen.correlated_mixture(1800, 3, seed=612)
    _lscv_check(kde, x3, oracle.grid_default(1800, 3, 16))
    grid, _ = kde.make_grid(n_h=128)
    _, g_default, h_default = kde.kde_lscv(dev(x), grid)
    _, g_explicit, _ = kde.kde_lscv(dev(x), _explicit(kde, h_default))
    assert np.array_equal(g_default, g_explicit)
    off = h.copy()
    off[37] *= 1 + 1e-9
    _lscv_check(kde, x, off)


@pytest.mark.parametrize("d,n,n_h", [(1, 3001, 128), (2, 2050, 256), (5, 1500, 96), (1, 700, 16 * 8)])
def test_octave_kernel_against_direct_kernel_and_oracle(kde, d, n, n_h):
    """On an octave grid (the default grid: n_h/8 points per octave of 1/h^2)
    the LSCV kernel squares exponentials down the octaves instead of calling
    ex2 for each; 8 bandwidths per thread keep the direct kernel.  Both against
    the oracle, and against each other."""
    x = datagen.correlated_mixture(n, d, seed=600 + d) if d > 1 else datagen.mixture_1d(n, seed=601)
    x64 = host64(x)
    h = oracle.grid_default(n, d, n_h)
    c = 1.0 / h ** 2
    P = n_h // 8
    assert np.allclose(c[:-P] / c[P:], 2.0, rtol=1e-12)
    grid, _ = kde.make_grid(n_h=n_h)
    res_o, g_o, hh = kde.kde_lscv(dev(x), grid)                                       # octave kernel
    res_d, g_d, _ = kde.kde_lscv(dev(x), grid, kde.make_opts(bw_per_thread=8))        # direct kernel
    assert np.allclose(hh, h, rtol=1e-14)
    ref = oracle.lscv_h(x64, h)
    A = lscv_A(x64)
    for g in (g_o, g_d):
        assert g_err(g, ref["g"], ref["s_kk"], ref["s_k"], h, n, d, A).max() < TOL
    assert g_err(g_o, g_d, ref["s_kk"], ref["s_k"], h, n, d, A).max() < TOL
    tiles = kde.kde_tile_count(n, 128 if n > 2048 else 32)
    s1, s2 = kde.kde_lscv_tile_sums(dev(x), h, 0, tiles)
    npairs = n * (n - 1) // 2
    assert s_err(s1, ref["s_kk"], npairs).max() < TOL
    assert s_err(s2, ref["s_k"], npairs).max() < TOL


def test_largest_grid_octave_kernel(kde):
    """The largest grid (1,024 points, 128 per octave of 1/h^2) on the octave
    kernel, against the oracle."""
    n, d = 1500, 1
    x = datagen.mixture_1d(n, seed=611)
    x64 = host64(x)
    h = oracle.grid_default(n, d, 1024)
    res, g, hh = kde.kde_lscv(dev(x), kde.make_grid(n_h=1024)[0])
    assert np.allclose(hh, h, rtol=1e-14)
    ref = oracle.lscv_h(x64, h)
    assert g_err(g, ref["g"], ref["s_kk"], ref["s_k"], h, n, d, lscv_A(x64)).max() < TOL
    assert argmin_ok(res["argmin"], ref["g"], TOL * np.max(np.abs(ref["g"])))


@pytest.mark.parametrize("log2_end,top", [(19.9, True), (21.0, True), (-19.9, False), (-21.0, False)])
def test_octave_grids_at_the_ends_of_the_exponent_add_range(kde, log2_end, top):
    """Octave-shaped grids (4 points per octave of 1/h^2) whose largest (top)
    or smallest h sits just inside or just outside [2^-20, 2^20]: inside, the
    octave kernel forms two of its three arguments by exponent adds and masks
    pairs with a finite squared distance (at h near 2^20 every real term is
    about 1 and a masked pair that leaked would add 1); outside, the direct
    kernel runs.  Both against the oracle (Eq. LSCV-gh).  At the small end
    the samples are evenly spaced (every pair at least 1.6e-3 sigma apart):
    near-duplicates of random samples would put g at the mercy of the FP32
    rounding of their whitened coordinates (h ~ 1e-6 sigma), a limit of the
    FP32 pair path rather than of the kernel's arithmetic."""
    n, d, n_h, P = 2100, 1, 16, 4
    x = datagen.mixture_1d(n, seed=612) if top else \
        datagen.rng(613).permutation(np.arange(n, dtype=np.float64))[None, :]
    x64 = host64(x)
    k = np.arange(n_h)
    expo = log2_end - (n_h - 1 - k) / (2.0 * P) if top else log2_end + k / (2.0 * P)
    h = 2.0 ** expo
    res, g, hh = kde.kde_lscv(dev(x), _explicit(kde, h))
    ref = oracle.lscv_h(x64, h)
    assert g_err(g, ref["g"], ref["s_kk"], ref["s_k"], h, n, d, lscv_A(x64)).max() < TOL
    s1, s2 = kde.kde_lscv_tile_sums(dev(x), h, 0, kde.kde_tile_count(n, kde.kde_item_tiles(n, d, n_h)["lscv_tile"]))
    npairs = n * (n - 1) // 2
    assert s_err(s1, ref["s_kk"], npairs).max() < TOL
    assert s_err(s2, ref["s_k"], npairs).max() < TOL
    if top:
        assert np.all(s1 <= npairs * (1 + 1e-6))  # no masked pair counted
