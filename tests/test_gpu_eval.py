"""Parity of the bandwidth consumers with the FP64 oracle: the density
estimate at query points (Sec. 4.2) and the range Count / Sum (Sec. 4.3).

Error metrics.  kde_eval: every pair term is one FP32 exp2 of a whitened
squared distance Q' (about 0.72 Mahalanobis^2); rounding of the whitened
coordinates (magnitude R) moves Q' by about 2 sqrt(Q') R 2^-24, a relative
term error below 1e-5 for the terms that carry the sum.  The error of f is
taken relative to max(f, 1e-3 max f) so that queries far in the tails, whose
few surviving terms have large Q', do not dominate.  kde_aqp: each term is a
normal-cdf difference in FP32 (absolute error about 2^-22); the count error is
bounded by TOL |count| + 2^-20 n, the sum error by TOL |sum| + 2^-20 n max|x|.
"""
import numpy as np
import pytest

import oracle
from paper_1505_01998_gb300 import datagen
from tests._helpers import TOL, built_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kde():
    return built_lib()


def dev(a, dtype="float32"):
    import torch
    a = np.ascontiguousarray(np.asarray(a))
    if a.ndim == 1:
        a = a[None, :]
    return torch.from_numpy(a.astype(dtype)).cuda()


def same(a, dtype="float32"):
    """The values the device sees, widened back to FP64 for the oracle."""
    a = np.asarray(a)
    if a.ndim == 1:
        a = a[None, :]
    return a.astype(dtype).astype(np.float64)


def f_err(got, ref):
    ref = np.asarray(ref)
    return np.abs(np.asarray(got) - ref) / np.maximum(ref, 1e-3 * ref.max())


def lscv_H_of(x64, h):
    _, S = oracle.mean_cov(x64)
    return h * h * S


# ------------------------------------------------------------- kde_eval

@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_eval_univariate_ragged(kde, dtype):
    n, m = 3001, 517
    x = datagen.mixture_1d(n, seed=11)
    x64 = same(x, dtype)
    q = np.linspace(x64.min() - 1.0, x64.max() + 1.0, m)[None, :]
    q64 = same(q, dtype)
    H = lscv_H_of(x64, 0.3)
    f = kde.kde_eval(dev(x, dtype), H, dev(q, dtype))
    ref = oracle.kde_eval(x64, H, q64)
    assert f_err(f, ref).max() < TOL


@pytest.mark.parametrize("d", [2, 3, 4, 5, 8, 12, 16])
def test_eval_multivariate(kde, d):
    n, m = 2017, 300
    x = datagen.correlated_mixture(n, d, seed=20 + d)
    x64 = same(x)
    g = datagen.rng(40 + d)
    # queries: samples moved by about one bandwidth, plus points in the tails
    q = x[:, :m].astype(np.float64) + 0.3 * g.standard_normal((d, m))
    q[:, -20:] = 3.0 * g.standard_normal((d, 20)) * x64.std(axis=1, keepdims=True)
    q64 = same(q)
    H = lscv_H_of(x64, 0.5)
    f = kde.kde_eval(dev(x), H, dev(q))
    ref = oracle.kde_eval(x64, H, q64)
    assert f_err(f, ref).max() < TOL


def test_eval_general_H_and_edge_sizes(kde):
    """A bandwidth matrix unrelated to S; n = 2; one query; queries equal to
    the samples; more queries than samples."""
    g = datagen.rng(7)
    d = 3
    H = datagen.random_spd(d, g, cond=20.0) * 0.05
    H = 0.5 * (H + H.T)  # exactly symmetric, as the entry point requires
    x = datagen.correlated_mixture(700, d, seed=8)
    x64 = same(x)
    for q in (x[:, :1], x, np.concatenate([x, x + 0.01], axis=1)):
        q64 = same(q)
        f = kde.kde_eval(dev(x), H, dev(q))
        assert f_err(f, oracle.kde_eval(x64, H, q64)).max() < TOL
    two = np.array([[0.0, 1.0]])
    f = kde.kde_eval(dev(two), [[0.25]], dev(np.array([[0.5, -3.0, 7.0]])))
    assert f_err(f, oracle.kde_eval(two, [[0.25]], np.array([[0.5, -3.0, 7.0]]))).max() < TOL


def test_eval_deterministic(kde):
    x = datagen.correlated_mixture(5000, 2, seed=3)
    H = lscv_H_of(same(x), 0.4)
    xd, qd = dev(x), dev(x[:, ::7])
    a = kde.kde_eval(xd, H, qd)
    b = kde.kde_eval(xd, H, qd)
    assert np.array_equal(a, b)


def test_eval_full_size_column(kde):
    """n = 65,536 skewed column with its plug-in bandwidth: queries every h/5
    over the range; sampled queries against the oracle; the estimate
    integrates to 1."""
    n = 65536
    x = datagen.skewed_column(n, seed=2)
    xd = dev(x)
    x64 = same(x)
    h = kde.kde_plugin(xd)["h"]
    lo, hi = x64.min() - 8 * h, x64.max() + 8 * h
    m = int(min(1 << 20, max(4096, np.ceil((hi - lo) / (0.2 * h)))))
    q = np.linspace(lo, hi, m)[None, :]
    f = kde.kde_eval(xd, [[h * h]], dev(q))
    idx = np.linspace(0, m - 1, 64).astype(np.int64)
    ref = oracle.kde_eval(x64, [[h * h]], same(q)[:, idx])
    assert f_err(f[idx], ref).max() < TOL
    # trapezoid rule on a grid finer than h / 5
    t = q[0]
    assert (t[1] - t[0]) <= 0.2 * h
    assert abs(float(np.sum(0.5 * (f[1:] + f[:-1]) * np.diff(t))) - 1.0) < 1e-3


def test_eval_errors(kde):
    x = dev(datagen.mixture_1d(100, seed=1))
    q = dev(np.zeros((1, 4)))
    with pytest.raises(kde.KdeError) as e:
        kde.kde_eval(x, [[-1.0]], q)
    assert e.value.status == kde.KDE_EDEGENERATE
    x2 = dev(datagen.correlated_mixture(100, 2, seed=1))
    with pytest.raises(kde.KdeError) as e:
        kde.kde_eval(x2, [[1.0, 0.5], [0.4, 1.0]], dev(np.zeros((2, 4))))
    assert e.value.status == kde.KDE_EINVAL
    with pytest.raises(kde.KdeError) as e:
        kde.kde_eval(x, [[np.nan]], q)
    assert e.value.status == kde.KDE_EINVAL
    need = kde.kde_eval_workspace_size(100, 1, 4)
    with pytest.raises(kde.KdeError) as e:
        kde.kde_eval(x, [[0.1]], q, ws=kde.workspace(need - 256))
    assert e.value.status == kde.KDE_ENOMEM
    # still usable
    f = kde.kde_eval(x, [[0.1]], q)
    assert np.all(np.isfinite(f))


# --------------------------------------------------------------- kde_aqp

def aqp_ok(kde, x, h, lo, hi, dtype="float32"):
    x64 = same(x, dtype)[0]
    c, s = kde.kde_aqp(dev(x, dtype), h, lo, hi)
    rc, rs = oracle.aqp(x64, h, np.float32(lo).astype(np.float64), np.float32(hi).astype(np.float64))
    n = x64.size
    amax = np.abs(x64).max()
    assert np.all(np.abs(c - rc) <= TOL * np.abs(rc) + 2.0 ** -20 * n), np.abs(c - rc).max()
    assert np.all(np.abs(s - rs) <= TOL * np.abs(rs) + 2.0 ** -20 * n * amax), np.abs(s - rs).max()
    return c, s


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_aqp_ranges(kde, dtype):
    n = 20011
    x = datagen.skewed_column(n, seed=5)
    x64 = same(x, dtype)[0]
    g = datagen.rng(9)
    span = x64.max() - x64.min()
    lo = x64.min() + g.uniform(-0.1, 1.0, 37) * span
    width = span * np.concatenate([g.uniform(0, 0.02, 12), g.uniform(0.02, 0.5, 20), [0, 0, 2, 5, 10]])
    hi = lo + width
    aqp_ok(kde, x, 0.05 * x64.std(), lo, hi, dtype)


def test_aqp_whole_line_and_empty_ranges(kde):
    x = datagen.mixture_1d(5000, seed=4)
    x64 = same(x)[0]
    lo = np.array([-np.inf, 0.3, 1.0, -np.inf, 50.0])
    hi = np.array([np.inf, 0.3, np.inf, 1.0, np.inf])
    c, s = kde.kde_aqp(dev(x), 0.2, lo, hi)
    assert abs(c[0] - x64.size) < 2.0 ** -20 * x64.size
    assert abs(s[0] - x64.sum()) < 1e-5 * np.abs(x64).sum()
    assert c[1] == 0.0 and s[1] == 0.0
    # complementary half-lines add up to the whole line
    assert abs(c[2] + c[3] - x64.size) < 1e-5 * x64.size
    assert abs(s[2] + s[3] - x64.sum()) < 1e-5 * np.abs(x64).sum()
    assert 0.0 <= c[4] < 1e-30


def test_aqp_full_size(kde):
    """4,194,304 samples, 64 ranges: every CTA holds several thousand samples."""
    n = 1 << 22
    x = datagen.skewed_column(n, seed=12)
    x64 = same(x)[0]
    g = datagen.rng(13)
    lo = np.quantile(x64, g.uniform(0, 0.9, 64))
    hi = lo + g.uniform(0, 1.0, 64) * x64.std()
    aqp_ok(kde, x, 0.02 * x64.std(), lo, hi)


@pytest.mark.parametrize("n", [2, 300, 456000, 912000])
def test_aqp_chunk_sizes(kde, n):
    """Sizes whose per-CTA chunks take each sort path on a 152-SM GPU: the
    shared-memory network (2 .. 1,024 keys) and the register-stage network
    with 8 and 16 keys per thread (2,048 and 4,096 keys per chunk)."""
    x = datagen.mixture_1d(n, seed=40 + n % 97)
    x64 = same(x)[0]
    g = datagen.rng(41)
    lo = np.quantile(x64, g.uniform(0, 1, 24)) - 0.5
    hi = lo + g.uniform(0, 3, 24)
    aqp_ok(kde, x, 0.15, lo, hi)


def test_aqp_many_ranges(kde):
    """The maximum number of ranges (1,024) over a small column."""
    x = datagen.mixture_1d(3000, seed=44)
    x64 = same(x)[0]
    g = datagen.rng(45)
    lo = g.uniform(x64.min() - 1, x64.max(), 1024)
    hi = lo + g.uniform(0, 2, 1024)
    aqp_ok(kde, x, 0.2, lo, hi)


def test_aqp_errors(kde):
    x = dev(datagen.mixture_1d(100, seed=1))
    for lo, hi, h in (([1.0], [0.0], 0.1), ([np.nan], [1.0], 0.1), ([0.0], [1.0], 0.0)):
        with pytest.raises(kde.KdeError) as e:
            kde.kde_aqp(x, h, lo, hi)
        assert e.value.status == kde.KDE_EINVAL
    need = kde.kde_aqp_workspace_size(100, 3)
    with pytest.raises(kde.KdeError) as e:
        kde.kde_aqp(x, 0.1, [0, 1, 2], [1, 2, 3], ws=kde.workspace(need - 256))
    assert e.value.status == kde.KDE_ENOMEM
