"""C ABI and host logic of libgbkde (CPU only: no kernel is launched)."""
import ctypes
import decimal
import math
import os
import re

import numpy as np
import pytest

import oracle
from tests._helpers import ROOT, built_lib


@pytest.fixture(scope="module")
def kde():
    return built_lib()


def _declared_functions():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(kde_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_function(kde):
    names = _declared_functions()
    assert len(names) >= 15
    L = kde.lib()
    for n in names:
        assert hasattr(L, n), f"{n} declared in include/ but not exported"
    # the Python binding covers the same names
    assert set(names) <= set(kde.SIGNATURES), set(names) - set(kde.SIGNATURES)


def test_version_and_status_strings(kde):
    assert "sm_103a" in kde.kde_version()
    L = kde.lib()
    for s in range(0, 11):
        assert L.kde_status_string(s)


def test_tile_map_exhaustive_against_column_enumeration(kde):
    # Column l holds l+1 tiles (Appendix A): enumerate columns and rows and
    # compare with the library's map for every tile number below 200k.
    L = kde.lib()
    lv, qv = ctypes.c_int64(), ctypes.c_int64()
    bx = 0
    for l in range(0, 632):
        for q in range(0, l + 1):
            assert L.kde_tile_coords(bx, ctypes.byref(lv), ctypes.byref(qv)) == 0
            assert (lv.value, qv.value) == (l, q), bx
            bx += 1


def test_tile_map_large_indices(kde):
    rng = np.random.default_rng(0)
    for l in list(rng.integers(1, 3_000_000, size=3000)) + [2**20 - 1, 2**24, 2**24 + 1, 3_999_999]:
        l = int(l)
        first = l * (l + 1) // 2
        for bx, q in ((first, 0), (first + l, l), (first + l // 2, l // 2)):
            assert kde.kde_tile_coords(bx) == (l, q)


def _walk_items(n, T, K):
    """Replay the kernels' tile walk (items of K consecutive tiles, stepping
    q -> q+1 and wrapping to the next column) and count pair visits."""
    tiles = kde_mod.kde_tile_count(n, T)
    seen = np.zeros((n, n), dtype=np.int32)
    for row in range((tiles + K - 1) // K):
        t0, t1 = row * K, min(row * K + K, tiles)
        l, q = kde_mod.kde_tile_coords(t0)
        for _t in range(t0, t1):
            for i in range(q * T, q * T + T):
                for j in range(l * T, l * T + T):
                    if i < j < n:
                        seen[i, j] += 1
            q += 1
            if q > l:
                l, q = l + 1, 0
    return seen


kde_mod = None


@pytest.mark.parametrize("n,T,K", [(97, 32, 1), (97, 32, 3), (130, 64, 2), (256, 32, 7), (33, 32, 5)])
def test_tile_walk_covers_each_pair_once(kde, n, T, K):
    global kde_mod
    kde_mod = kde
    seen = _walk_items(n, T, K)
    iu = np.triu_indices(n, 1)
    assert np.all(seen[iu] == 1)
    assert seen.sum() == n * (n - 1) // 2


def test_default_grid_matches_oracle(kde):
    for n, d in ((1024, 1), (65536, 1), (16384, 3)):
        assert np.allclose(kde.kde_default_grid(n, d, 128), oracle.grid_default(n, d, 128), rtol=1e-14)


def test_workspace_size_monotone_and_bad_args(kde):
    a = kde.kde_workspace_size(1000, 1, 64)
    b = kde.kde_workspace_size(100000, 1, 64)
    assert 0 < a < b
    with pytest.raises(kde.KdeError) as e:
        kde.kde_workspace_size(1, 1, 64)
    assert e.value.status == kde.KDE_EINVAL
    with pytest.raises(kde.KdeError):
        kde.kde_workspace_size(100, 17, 64)
    with pytest.raises(kde.KdeError):
        kde.kde_workspace_size(100, 1, 64, kde.make_opts(tile=48))


def test_bandwidths_per_thread_options(kde):
    """2, 8 and 16 bandwidths per thread are accepted; anything else is an
    argument error before any launch."""
    for b in (0, 2, 8, 16):
        assert kde.kde_workspace_size(3000, 4, 64, kde.make_opts(bw_per_thread=b)) > 0
    for b in (1, 4, 12, 32):
        with pytest.raises(kde.KdeError) as e:
            kde.kde_workspace_size(3000, 4, 64, kde.make_opts(bw_per_thread=b))
        assert e.value.status == kde.KDE_EINVAL


def test_double_float_butterfly_replayed_on_the_host():
    """The item totals of the pair kernels are warp sums of FP32 (hi, lo) pairs
    by a butterfly with Knuth's TwoSum at each step and Dekker's Fast2Sum to
    renormalise (warp_sum_ff).  Replayed here in numpy float32 with the same
    operation order: every lane ends with the same pair (the steps are
    symmetric), and the pair carries the exact sum to about 44 bits."""
    f = np.float32
    rng = np.random.default_rng(5)
    for trial in range(200):
        scale = 10.0 ** rng.uniform(-6, 9)
        hi = (rng.lognormal(0, 2, 32) * scale).astype(f)
        lo = (hi * rng.uniform(-1, 1, 32) * 2.0 ** -25).astype(f)  # Kahan tails: below an ulp of hi
        h, l = hi.copy(), lo.copy()
        o = 16
        while o:
            idx = np.arange(32) ^ o
            h2, l2 = h[idx], l[idx]
            s = f(h + h2)
            bb = f(s - h)
            e = f(f(h - f(s - bb)) + f(h2 - bb))
            t = f(f(l + l2) + e)
            h = f(s + t)
            l = f(t - f(h - s))
            o >>= 1
        assert np.all(h == h[0]) and np.all(l == l[0])
        exact = math.fsum([float(v) for v in hi] + [float(v) for v in lo])
        got = float(h[0]) + float(l[0])
        assert abs(got - exact) <= 2.0 ** -43 * abs(exact), (trial, got, exact)


@pytest.mark.parametrize("K", [5, 7, 9])
def test_newton_root_replayed_on_the_host(K):
    """The PLUGIN chain's real roots (g2 = a^(1/7), h = b^(1/5)) are formed
    on the device by root_newton: x = m 2^(K q) with m in [1, 2^K) (the
    exponent split by floor division), an FP32 seed 2^(-log2(m) / K), two
    Newton steps w <- w + w (1 - m w^K) / K for w = m^(-1/K), then
    x^(1/K) = m w^(K-1) 2^q and x^(-1/K) = w 2^-q.  Replayed here in numpy
    FP64 with an FP32 seed perturbed by 2^-19 (looser than the MUFU seed):
    across the whole normal range and at exponents of every residue mod K,
    both results agree with the powers (40-digit decimal arithmetic) to a few
    ulp."""
    decimal.getcontext().prec = 40
    rng = np.random.default_rng(K)
    xs = np.concatenate([10.0 ** rng.uniform(-307, 308, 400), 2.0 ** np.arange(-1022, 1024, 37, dtype=np.float64),
                         [2.2250738585072014e-308, 1.7976931348623157e308, 1.0, 0.5, 3.0]])
    for x in xs:
        bits = int(np.float64(x).view(np.int64))
        e = ((bits >> 52) & 0x7FF) - 1023
        q, r = e // K, e % K
        m = float(np.int64((bits & 0x000FFFFFFFFFFFFF) | ((1023 + r) << 52)).view(np.float64))
        assert 1.0 <= m < 2.0 ** K and m * 2.0 ** (K * q) == x
        seed = np.float32(2.0 ** (-math.log2(float(np.float32(m))) / K)) * np.float32(1 + 2.0 ** -19)
        w = float(seed)
        for _ in range(2):
            t = 1.0 - m * w ** K
            w = w + w * t / K
        y = m * w ** (K - 1) * 2.0 ** q
        inv = w * 2.0 ** -q
        ref = float(decimal.Decimal(x) ** (decimal.Decimal(1) / decimal.Decimal(K)))
        assert abs(y - ref) <= 1.5e-15 * ref, (K, x, y, ref)
        assert abs(inv * ref - 1.0) <= 1.5e-15, (K, x, inv, ref)


def _ff_add(h, l, h2, l2):
    f = np.float32
    s = f(h + h2)
    bb = f(s - h)
    e = f(f(h - f(s - bb)) + f(h2 - bb))
    t = f(f(l + l2) + e)
    hn = f(s + t)
    return hn, f(t - f(hn - s))


@pytest.mark.parametrize("two_halves", [True, False])
def test_double_float_lane_order_sum_replayed_on_the_host(two_halves):
    """The Kahan-mode item totals of the LSCV kernel are warp sums of FP32
    (hi, lo) pairs taken by one lane per sum in a fixed, staggered lane order
    (warp_sums_ff_transposed): over all 32 lanes from lane q, or over two
    halves of 16 lanes whose totals are then added.  Replayed in numpy float32
    with the same order: the pair carries the exact sum to about 44 bits."""
    f = np.float32
    rng = np.random.default_rng(6)
    for trial in range(200):
        q = int(rng.integers(0, 16 if two_halves else 32))
        scale = 10.0 ** rng.uniform(-6, 9)
        hi = (rng.lognormal(0, 2, 32) * scale).astype(f)
        lo = (hi * rng.uniform(-1, 1, 32) * 2.0 ** -25).astype(f)
        parts = [range(0, 16), range(16, 32)] if two_halves else [range(32)]
        tot = []
        for lanes in parts:
            lanes = list(lanes)
            h, l = f(0), f(0)
            for i in range(len(lanes)):
                k = lanes[(i + q) % len(lanes)]
                h, l = _ff_add(h, l, hi[k], lo[k])
            tot.append((h, l))
        h, l = tot[0]
        if two_halves:
            h, l = _ff_add(h, l, *tot[1])
        exact = math.fsum([float(v) for v in hi] + [float(v) for v in lo])
        got = float(h) + float(l)
        assert abs(got - exact) <= 2.0 ** -43 * abs(exact), (trial, got, exact)


def test_clock_sample_summary():
    """The benchmark's summary of nvidia-smi samples taken during the timed
    region: idle samples (below half the highest clock) leave the median, and
    every throttle reason seen active is reported."""
    import bench
    idle = "0, 345, 2070, 120.5, 0x0, Not Active, Not Active, Not Active, Not Active\n"
    busy = "0, 2070, 2070, 340.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
    capped = "0, 1965, 2070, 1398.0, 0x4, Not Active, Not Active, Not Active, Active\n"
    hot = "0, 1800, 2070, 1200.0, 0x40, Not Active, Active, Not Active, Not Active\n"
    out = bench.parse_clock_samples([idle, busy, busy, capped, "garbage line\n"])
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["samples"] == 4 and out["power_w_max"] == 1398.0
    assert out["reasons"] == ["sw_power_cap"]
    out = bench.parse_clock_samples([busy, hot, capped])
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert out["sm_mhz"] == 1965.0
    assert bench.parse_clock_samples([]) is None


def test_entry_points_reject_bad_arguments_before_any_launch(kde):
    L = kde.lib()
    grid, keep = kde.make_grid(n_h=8)
    res = kde.kde_result()
    dummy = ctypes.c_void_p(256)  # never dereferenced: argument checks fail first
    # NULL samples
    assert L.kde_lscv(None, 0, 100, 1, ctypes.byref(grid), None, dummy, 1 << 20, None, None, None,
                      ctypes.byref(res)) == kde.KDE_EINVAL
    # d out of range
    assert L.kde_lscv(dummy, 0, 100, 17, ctypes.byref(grid), None, dummy, 1 << 20, None, None, None,
                      ctypes.byref(res)) == kde.KDE_EINVAL
    # n < 2
    assert L.kde_plugin(dummy, 0, 1, None, dummy, 1 << 20, None, ctypes.byref(res)) == kde.KDE_EINVAL
    # misaligned workspace
    assert L.kde_plugin(dummy, 0, 100, None, ctypes.c_void_p(260), 1 << 20, None,
                        ctypes.byref(res)) == kde.KDE_EINVAL
    # bad dtype
    assert L.kde_plugin(dummy, 7, 100, None, dummy, 1 << 20, None, ctypes.byref(res)) == kde.KDE_EINVAL
    # empty grid / too many bandwidths
    g0 = kde.kde_grid(kde.KDE_GRID_DEFAULT_Z, 0, None, 0.0, 0.0)
    assert L.kde_lscv(dummy, 0, 100, 1, ctypes.byref(g0), None, dummy, 1 << 20, None, None, None,
                      ctypes.byref(res)) == kde.KDE_EINVAL
    g2 = kde.kde_grid(kde.KDE_GRID_DEFAULT_Z, 2000, None, 0.0, 0.0)
    assert L.kde_lscv(dummy, 0, 100, 1, ctypes.byref(g2), None, dummy, 1 << 20, None, None, None,
                      ctypes.byref(res)) == kde.KDE_EINVAL
    g1025 = kde.kde_grid(kde.KDE_GRID_DEFAULT_Z, kde.KDE_MAX_NH + 1, None, 0.0, 0.0)
    assert L.kde_lscv(dummy, 0, 100, 1, ctypes.byref(g1025), None, dummy, 1 << 20, None, None, None,
                      ctypes.byref(res)) == kde.KDE_EINVAL
    # the merge steps of sharded selections check their arguments on the host
    assert L.kde_plugin_merge(1, 8, 1.0, ctypes.byref(res)) == kde.KDE_EINVAL
    assert L.kde_plugin_merge(100, 8, float("nan"), ctypes.byref(res)) == kde.KDE_EINVAL
    assert L.kde_item_tiles(100, 0, None, 8, None, None, None, None, None) == kde.KDE_EINVAL
    # a log grid with a non-positive bound
    g3 = kde.kde_grid(kde.KDE_GRID_LOG, 8, None, -1.0, 2.0)
    assert L.kde_lscv(dummy, 0, 100, 1, ctypes.byref(g3), None, dummy, 1 << 20, None, None, None,
                      ctypes.byref(res)) == kde.KDE_EINVAL
    buf = ctypes.create_string_buffer(256)
    assert L.kde_last_error(buf, 256) == kde.KDE_EINVAL
    assert b"grid" in buf.value


def test_oracle_and_library_share_no_code():
    """The oracle never imports the CUDA package and vice versa."""
    osrc = open(os.path.join(ROOT, "oracle", "__init__.py")).read() + \
        open(os.path.join(ROOT, "oracle", "kde_oracle.c")).read()
    assert "paper_1505_01998_gb300" not in osrc.replace("in ``paper_1505_01998_gb300``", "")
    pkg = os.path.join(ROOT, "paper_1505_01998_gb300")
    for dp, _, fs in os.walk(pkg):
        for f in fs:
            if f.endswith((".py", ".cu", ".cuh", ".hpp", ".cpp", ".h")):
                src = open(os.path.join(dp, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "kde_oracle" not in src, f


def test_autotune_cache_text_roundtrip(kde, tmp_path):
    p = tmp_path / "cache.txt"
    p.write_text("# header\nSomeGPU/152 1 1 7 14 128 16 2 1 9.1e12\nbad line\nSomeGPU/152 0 2 8 16 32 8 1 2 1e12\n")
    kde.kde_autotune_clear()
    kde.kde_autotune_load(p)
    q = tmp_path / "out.txt"
    kde.kde_autotune_save(q)
    lines = [l for l in q.read_text().splitlines() if not l.startswith("#")]
    assert len(lines) == 2 and any(l.startswith("SomeGPU/152 1 1 7 14 128 16 2 1") for l in lines)
    kde.kde_autotune_clear()
    with pytest.raises(kde.KdeError):
        kde.kde_autotune_load(tmp_path / "missing.txt")


def test_normal_tail_approximation_of_the_range_aggregates():
    """The upper normal tail used by kde_aqp (Hastings' rational approximation,
    Abramowitz & Stegun 7.1.26, absolute error 7.5e-8 in exact arithmetic),
    replayed in numpy FP32 with the constants read from the CUDA source:
    within 4e-7 of erfc(t/sqrt 2)/2 for every t (the FP32 rounding of 1 - q
    near 1 adds up to 6e-8)."""
    erfc = pytest.importorskip("scipy.special").erfc
    src = open(os.path.join(ROOT, "paper_1505_01998_gb300", "csrc", "eval.cu")).read()
    c = {k: np.float32(v) for k, v in re.findall(r"kAs(P|A\d) = (-?[0-9.]+)f", src)}
    assert sorted(c) == ["A1", "A2", "A3", "A4", "A5", "P"]
    t = np.linspace(-12.0, 12.0, 400_001).astype(np.float32)
    u = (np.abs(t) * np.float32(0.70710678118654752)).astype(np.float32)
    e = np.exp(-(u * u)).astype(np.float32)
    sd = (np.float32(1.0) / (c["P"] * u + np.float32(1.0))).astype(np.float32)
    poly = sd * (c["A1"] + sd * (c["A2"] + sd * (c["A3"] + sd * (c["A4"] + sd * c["A5"]))))
    q = (np.float32(0.5) * poly.astype(np.float32) * e).astype(np.float32)
    Q = np.where(t >= 0, q, np.float32(1.0) - q).astype(np.float64)
    ref = 0.5 * erfc(t.astype(np.float64) / np.sqrt(2.0))
    assert np.abs(Q - ref).max() < 4e-7


@pytest.mark.parametrize("R,RG", [(2, 1), (8, 1), (8, 2)])
def test_psi_edge_masks_in_tile_local_indices(R, RG):
    """The psi kernel masks the pairs of edge tiles (the diagonal and the
    ragged last column) by tile-local 32-bit indices: lane row
    il = il0 + 64 p (+ 32 for the second of a packed pair) with
    il0 = row-group offset + lane on a diagonal tile and -2^30 off it, column
    jl within the tile, kept when il < jl < jlim, jlim = min(T, n - l T).
    Replayed here for every lane, packed pair and column of the edge tiles of
    ragged sizes against the global rule i < j < n with i, j sample indices."""
    T = 32 * R * RG
    SL = 8 // RG
    for n in (T + 1, 2 * T - 7, 3 * T, 3 * T + 5):
        NT = (n + T - 1) // T
        for l in range(NT):
            for q in range(l + 1):
                edge = q == l or (l + 1) * T > n
                if not edge:
                    continue
                jlim = min(T, n - l * T)
                for warp in range(8):
                    rg = warp // SL
                    r0 = rg * 32 * R  # + lane below
                    for lane in range(32):
                        il0 = (r0 + lane) if q == l else -(1 << 30)
                        for p in range(R // 2):
                            for half in (0, 1):
                                il = il0 + 64 * p + 32 * half
                                i = q * T + r0 + lane + 64 * p + 32 * half
                                for jl in range(T):
                                    j = l * T + jl
                                    assert (il < jl < jlim) == (i < j < n), (n, l, q, warp, lane, p, half, jl)
