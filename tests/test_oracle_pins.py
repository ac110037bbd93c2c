"""Pins of the FP64 oracle against facts outside itself (CPU only).

Each test checks the oracle against something that does not share its formula
text: values the paper prints (tests/golden/paper_constants.json), symbolic
differentiation (sympy), library routines (numpy/scipy), quadrature, closed
forms, exact expectations, invariants and brute force on tiny inputs.  The
pins are chosen so that a plausible slip in the oracle -- a dropped term, a
wrong sign, index or power, a transposed operand -- fails at least one.
"""
import json
import math
import os

import numpy as np
import pytest
import sympy as sp
from numpy.polynomial import hermite_e
from scipy import integrate, stats

import oracle
from paper_1505_01998_gb300 import datagen

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


# ----------------------------------------------------------- constants

def test_kernel_derivative_constants_match_paper():
    assert oracle.gauss_deriv(6, 0.0) == pytest.approx(GOLD["K6_at_0"]["value"], rel=1e-15)
    assert oracle.gauss_deriv(4, 0.0) == pytest.approx(GOLD["K4_at_0"]["value"], rel=1e-15)


def test_hermite_matches_numpy_hermite_e():
    for r in range(0, 11):
        c = np.zeros(r + 1)
        c[r] = 1.0
        for x in (-3.7, -1.0, -0.2, 0.0, 0.5, 1.3, 2.9, 6.0):
            assert oracle.hermite(r, x) == pytest.approx(hermite_e.hermeval(x, c), rel=1e-13, abs=1e-12)


def test_paper_polynomials_are_the_recurrence():
    for key, r in (("K6_polynomial", 6), ("K4_polynomial", 4)):
        coeffs = GOLD[key]["coeffs_high_to_low"]
        for x in np.linspace(-5, 5, 23):
            assert oracle.hermite(r, x) == pytest.approx(np.polyval(coeffs, x), rel=1e-13, abs=1e-11)


def test_gauss_derivatives_match_sympy():
    xs = sp.symbols("x")
    phi = sp.exp(-xs ** 2 / 2) / sp.sqrt(2 * sp.pi)
    for r in range(0, 9):
        f = sp.lambdify(xs, sp.diff(phi, xs, r), "math")
        for x in (-4.1, -2.0, -0.7, 0.0, 0.3, 1.5, 3.3):
            assert oracle.gauss_deriv(r, x) == pytest.approx(f(x), rel=1e-12, abs=1e-15)


def _psi_normal_exact(r, sigma):
    """psi_r = int f^(r) f dx for f = N(0, sigma^2), by quadrature of the sympy
    derivative (independent of any closed form)."""
    xs = sp.symbols("x")
    f = sp.exp(-xs ** 2 / (2 * sigma ** 2)) / (sigma * sp.sqrt(2 * sp.pi))
    fr = sp.lambdify(xs, sp.diff(f, xs, r) * f, "math")
    val, _ = integrate.quad(fr, -40 * sigma, 40 * sigma, limit=400, epsabs=0, epsrel=1e-13)
    return val


@pytest.mark.parametrize("sigma", [0.4, 1.0, 2.7])
def test_psi8_normal_scale_is_the_normal_functional(sigma):
    assert oracle.psi8_ns(sigma) == pytest.approx(_psi_normal_exact(8, sigma), rel=1e-9)
    assert oracle.psi8_ns(1.0) == pytest.approx(GOLD["psi8_ns_coefficient"]["value"], rel=1e-15)


def test_plugin_final_step_gives_rule_of_thumb():
    # With psi4 replaced by its normal-scale value, Eq. PLUGIN-Final_h must give
    # h = (4/(3n))^(1/5) sigma (the normal-reference rule of thumb).
    for sigma in (0.3, 1.0, 5.0):
        for n in (100, 1024, 65536):
            psi4 = _psi_normal_exact(4, sigma)
            assert oracle.plugin_h(psi4, n) == pytest.approx((4.0 / (3 * n)) ** 0.2 * sigma, rel=1e-9)


def test_pilot_bandwidths_are_amse_optimal_form():
    # g1 and g2 are the AMSE-optimal pilots g = [2 K^(r)(0) / (-mu2 psi_{r+2} n)]^(1/(r+3))
    # for r = 6 and r = 4; at normal scale they equal known closed forms in sigma.
    for sigma in (0.5, 2.0):
        for n in (256, 4096):
            psi8 = _psi_normal_exact(8, sigma)
            psi6 = _psi_normal_exact(6, sigma)
            k6 = GOLD["K6_at_0"]["value"]
            k4 = GOLD["K4_at_0"]["value"]
            assert oracle.plugin_g1(psi8, n) == pytest.approx((2 * k6 / (-psi8 * n)) ** (1 / 9), rel=1e-12)
            assert oracle.plugin_g2(psi6, n) == pytest.approx((2 * k4 / (-psi6 * n)) ** (1 / 7), rel=1e-12)


def test_h0_matches_paper_constants_at_d1_and_normal_scale():
    for n in (64, 1024, 65536):
        d = 1
        ratio = 1.0 / (2 ** d * math.pi ** (d / 2) * d ** 2)
        rf2 = d * (d + 2) / (2 ** (d + 2) * math.pi ** (d / 2))
        lit = (ratio / (rf2 * n)) ** (1 / (d + 4))
        assert oracle.h0(n, 1) == pytest.approx(lit, rel=1e-14)
        for d in (2, 3, 4):
            assert oracle.h0(n, d) == pytest.approx((4.0 / ((d + 2) * n)) ** (1 / (d + 4)), rel=1e-14)


def test_default_grid_spans_search_range():
    """Log-spaced over Z(h0) = [h0/4, 4 h0) (Eq. LSCV-Zh0): first point at the
    lower end, the step one n_h-th of the range's log-width, so the point after
    the last is the upper end; with n_h a multiple of 8, 1/h^2 halves every
    n_h/8 points."""
    g = oracle.grid_default(1000, 1, 150)
    z = oracle.h0(1000, 1)
    assert g[0] == pytest.approx(z * GOLD["search_range"]["lo_factor"], rel=1e-14)
    step = np.log(GOLD["search_range"]["hi_factor"] / GOLD["search_range"]["lo_factor"]) / 150
    assert np.allclose(np.diff(np.log(g)), step, rtol=1e-12)
    assert g[-1] * np.exp(step) == pytest.approx(z * GOLD["search_range"]["hi_factor"], rel=1e-13)
    g = oracle.grid_default(65536, 1, 256)
    c = 1.0 / g ** 2
    assert np.allclose(c[:-32] / c[32:], 2.0, rtol=1e-13)


def test_log_grid_endpoints_and_constant_ratio():
    """n_h points from h_min to h_max, both ends included, each step the same
    ratio (h_max/h_min)^(1/(n_h-1)); the 64-point grid over [0.01, 2] of the
    n = 1,024 mixture workload steps by 1.0877 (200^(1/63)).  Checked against
    numpy's geometric spacing and the closed-form ratio."""
    for lo, hi, n_h in ((0.01, 2.0, 64), (0.3, 0.31, 7), (1e-3, 1e3, 256), (2.0, 0.5, 5)):
        g = oracle.grid_log(lo, hi, n_h)
        assert g.size == n_h
        assert g[0] == lo
        assert g[-1] == pytest.approx(hi, rel=1e-14)
        ratio = (hi / lo) ** (1.0 / (n_h - 1))
        assert np.allclose(g[1:] / g[:-1], ratio, rtol=1e-13)
        assert np.allclose(g, np.geomspace(lo, hi, n_h), rtol=1e-13)
    g = oracle.grid_log(0.01, 2.0, 64)
    assert g[1] / g[0] == pytest.approx(1.0877, abs=5e-5)
    assert np.all(np.diff(g) > 0)


def test_log_grid_single_point_is_the_lower_end():
    assert list(oracle.grid_log(0.25, 4.0, 1)) == [0.25]
    assert list(oracle.grid_log(0.7, 0.7, 3)) == [0.7, 0.7, 0.7]


# ------------------------------------------------------------- stats

def test_mean_cov_and_inverse_match_numpy():
    x = datagen.correlated_mixture(500, 3, seed=11).astype(np.float64)
    m, c = oracle.mean_cov(x)
    assert np.allclose(m, x.mean(axis=1), rtol=1e-13, atol=1e-13)
    assert np.allclose(c, np.cov(x), rtol=1e-12)
    ci, det, rc = oracle.invert(c)
    assert rc == 0
    assert np.allclose(ci, np.linalg.inv(c), rtol=1e-11)
    assert det == pytest.approx(np.linalg.det(c), rel=1e-12)


# -------------------------------------------------------- psi sums

def _psi_bruteforce(x, r, g):
    """Full i != j double sum with numpy's HermiteE, different loop order."""
    x = np.asarray(x, dtype=np.float64).ravel()
    n = x.size
    c = np.zeros(r + 1)
    c[r] = 1.0
    tot = 0.0
    for j in range(n - 1, -1, -1):
        for i in range(n):
            if i == j:
                continue
            u = (x[i] - x[j]) / g
            tot += hermite_e.hermeval(u, c) * math.exp(-u * u / 2) / math.sqrt(2 * math.pi)
    return tot


@pytest.mark.parametrize("r", [4, 6, 8])
@pytest.mark.parametrize("n", [2, 7, 33, 64])
def test_psi_pair_sum_bruteforce(r, n):
    x = datagen.mixture_1d(n, seed=100 + n)[0]
    g = 0.37
    full = _psi_bruteforce(x, r, g)
    assert 2 * oracle.psi_pair_sum(x, r, g) == pytest.approx(full, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("r", [4, 6])
def test_psi_n2_closed_form(r):
    x = np.array([0.3, 1.1])
    g = 0.8
    k = lambda u: oracle.gauss_deriv(r, u)
    expect = (k((x[0] - x[1]) / g) + k(0.0)) / (2 * g ** (r + 1))
    assert oracle.psi(x, r, g) == pytest.approx(expect, rel=1e-14)


@pytest.mark.parametrize("r", [4, 6])
def test_psi_exact_expectation_for_normal_samples(r):
    # E psi_r(g) = ((n-1)/n) s^-(r+1) K^(r)(0) + n^-1 g^-(r+1) K^(r)(0), s^2 = g^2 + 2 sigma^2.
    n, sigma, g, reps = 40, 1.3, 0.6, 400
    rng = datagen.rng(7 + r)
    vals = np.array([oracle.psi(rng.normal(0.0, sigma, n), r, g, threads=1) for _ in range(reps)])
    k0 = oracle.gauss_deriv(r, 0.0)
    s = math.sqrt(g * g + 2 * sigma * sigma)
    expect = (n - 1) / n * s ** (-(r + 1)) * k0 + g ** (-(r + 1)) * k0 / n
    se = vals.std(ddof=1) / math.sqrt(reps)
    assert abs(vals.mean() - expect) < 4 * se


def test_psi_invariances():
    x = datagen.mixture_1d(300, seed=5)[0]
    rng = datagen.rng(9)
    for r in (4, 6):
        p = oracle.psi(x, r, 0.5)
        assert oracle.psi(rng.permutation(x), r, 0.5) == pytest.approx(p, rel=1e-12)
        assert oracle.psi(x + 17.25, r, 0.5) == pytest.approx(p, rel=1e-9)
        a = 3.5
        assert oracle.psi(a * x, r, a * 0.5) == pytest.approx(a ** (-(r + 1)) * p, rel=1e-11)


def test_psi_block_decomposition_adds_up():
    x = datagen.skewed_column(200, seed=3)[0].astype(np.float64)
    full = oracle.psi_pair_sum(x, 6, 7.0)
    cuts = [0, 37, 64, 150, 200]
    tot = 0.0
    for a in range(4):
        for b in range(a, 4):
            tot += oracle.psi_pair_sum(x, 6, 7.0, block=(cuts[a], cuts[a + 1], cuts[b], cuts[b + 1]))
    assert tot == pytest.approx(full, rel=1e-12)


def _psi_abs_block_bruteforce(x, r, g, i0, i1, j0, j1):
    """sum of |He_r(u) phi(u)| over i in [i0,i1), j in [j0,j1), i < j, built as a
    numpy mask over the full difference matrix (no loop shared with the oracle)."""
    x = np.asarray(x, dtype=np.float64).ravel()
    n = x.size
    c = np.zeros(r + 1)
    c[r] = 1.0
    u = (x[:, None] - x[None, :]) / g
    t = np.abs(hermite_e.hermeval(u, c) * np.exp(-u * u / 2) / math.sqrt(2 * math.pi))
    i = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    mask = (i < j) & (i >= i0) & (i < i1) & (j >= j0) & (j < j1)
    return float(t[mask].sum())


@pytest.mark.parametrize("r", [4, 6])
@pytest.mark.parametrize("n", [2, 9, 40, 64])
def test_psi_abs_pair_sum_bruteforce(r, n):
    """The magnitude scale that every psi tolerance divides by: each unordered
    pair once (not twice, not i = j), |.| taken per term."""
    x = datagen.mixture_1d(n, seed=300 + n)[0]
    for g in (0.15, 0.6, 3.0):
        ref = _psi_abs_block_bruteforce(x, r, g, 0, n, 0, n)
        assert oracle.psi_abs_pair_sum(x, r, g) == pytest.approx(ref, rel=1e-12, abs=1e-300)
        # the full i != j sum of |terms| is exactly twice the i < j one
        full = _psi_bruteforce_abs(x, r, g)
        assert 2 * oracle.psi_abs_pair_sum(x, r, g) == pytest.approx(full, rel=1e-12)
    if n >= 40:
        for blk in ((0, 13, 0, 40), (5, 21, 17, 40), (30, 40, 0, 10), (0, n, 33, 34)):
            ref = _psi_abs_block_bruteforce(x, r, 0.6, *blk)
            got = oracle.psi_abs_pair_sum(x, r, 0.6, block=blk)
            assert got == pytest.approx(ref, rel=1e-12, abs=1e-300), blk


def _psi_bruteforce_abs(x, r, g):
    x = np.asarray(x, dtype=np.float64).ravel()
    c = np.zeros(r + 1)
    c[r] = 1.0
    tot = 0.0
    for j in range(x.size - 1, -1, -1):
        for i in range(x.size):
            if i != j:
                u = (x[i] - x[j]) / g
                tot += abs(hermite_e.hermeval(u, c)) * math.exp(-u * u / 2) / math.sqrt(2 * math.pi)
    return tot


def test_psi_abs_pair_sum_bounds_the_signed_sum_with_equality_for_one_sign():
    """sum |t| >= |sum t| always.  Equality when every term has one sign:
    He_6 < 0 on |u| < 0.6167 (its smallest positive root), so samples packed
    within half a bandwidth give only negative K^(6) terms; He_4 > 0 for
    |u| > 2.3344 (its largest root), so samples spaced three bandwidths apart
    give only positive K^(4) terms."""
    x = datagen.skewed_column(300, seed=8)[0].astype(np.float64)
    for r in (4, 6):
        for g in (0.5, 4.0, 30.0):
            s = oracle.psi_pair_sum(x, r, g)
            a = oracle.psi_abs_pair_sum(x, r, g)
            assert a >= abs(s) * (1 - 1e-14)
            assert a > 1.5 * abs(s)  # mixed signs at these bandwidths
    rng = datagen.rng(12)
    packed = rng.uniform(0.0, 0.5, 50)  # every |u| < 0.5 at g = 1
    s6 = oracle.psi_pair_sum(packed, 6, 1.0)
    assert s6 < 0
    assert oracle.psi_abs_pair_sum(packed, 6, 1.0) == pytest.approx(-s6, rel=1e-14)
    spaced = 3.0 * np.arange(40) + rng.uniform(0, 0.1, 40)  # every |u| > 2.9 at g = 1
    s4 = oracle.psi_pair_sum(spaced, 4, 1.0)
    assert s4 > 0
    assert oracle.psi_abs_pair_sum(spaced, 4, 1.0) == pytest.approx(s4, rel=1e-14)


# ------------------------------------------------------------ plug-in

def test_plugin_chain_is_consistent_and_equivariant():
    x = datagen.mixture_1d(400, seed=21)[0]
    p = oracle.plugin(x)
    assert p["status"] == 0
    assert p["sigma"] == pytest.approx(np.std(x, ddof=1), rel=1e-13)
    assert p["psi6"] == pytest.approx(oracle.psi(x, 6, p["g1"]), rel=1e-14)
    assert p["g2"] == pytest.approx(oracle.plugin_g2(p["psi6"], x.size), rel=1e-14)
    assert p["psi4"] == pytest.approx(oracle.psi(x, 4, p["g2"]), rel=1e-14)
    a = 0.01
    q = oracle.plugin(a * x - 3.0)
    assert q["h"] == pytest.approx(a * p["h"], rel=1e-10)


def test_plugin_approaches_rule_of_thumb_for_normal_data():
    n = 3000
    hs = []
    for s in range(6):
        x = datagen.rng(300 + s).normal(0.0, 2.0, n)
        hs.append(oracle.plugin(x)["h"] / np.std(x, ddof=1))
    assert np.mean(hs) == pytest.approx((4.0 / (3 * n)) ** 0.2, rel=0.06)


def test_plugin_degenerate_inputs():
    assert oracle.plugin(np.ones(10))["status"] == oracle.EDEGENERATE
    assert oracle.plugin(np.ones(1))["status"] == oracle.EINVAL


# ------------------------------------------------------------- LSCV_h

def _lscv_d1_by_quadrature(x, h):
    """g(h) = int fhat^2 - 2 n^-2 sum_{i != j} K_H(X_i - X_j) with H = h^2 sigma^2:
    the integral of the squared estimate is done numerically, independent of the
    K*K closed form."""
    x = np.asarray(x, dtype=np.float64).ravel()
    n = x.size
    bw = h * np.std(x, ddof=1)
    fhat = lambda t: np.sum(stats.norm.pdf(t, loc=x, scale=bw)) / n
    pts = np.sort(x)
    lo, hi = pts[0] - 12 * bw, pts[-1] + 12 * bw
    val, _ = integrate.quad(lambda t: fhat(t) ** 2, lo, hi, points=pts, limit=2000,
                            epsabs=0, epsrel=1e-12)
    cross = 0.0
    for i in range(n):
        for j in range(n):
            if i != j:
                cross += stats.norm.pdf(x[i] - x[j], scale=bw)
    return val - 2.0 * cross / n ** 2


@pytest.mark.parametrize("seed", [1, 2])
def test_lscv_d1_matches_quadrature(seed):
    x = datagen.mixture_1d(12, seed=seed)[0]
    h = np.array([0.05, 0.2, 0.5, 1.3])
    g = oracle.lscv_h(x, h)["g"]
    for k in range(h.size):
        assert g[k] == pytest.approx(_lscv_d1_by_quadrature(x, h[k]), rel=1e-8, abs=1e-12)


def _lscv_mvn_bruteforce(x, h):
    """g(h) at H = h^2 S from scipy's multivariate normal densities:
    2 n^-2 sum_{i<j} [N(v; 0, 2H) - 2 N(v; 0, H)] + n^-1 N(0; 0, 2H)."""
    x = np.asarray(x, dtype=np.float64)
    d, n = x.shape
    S = np.cov(x)
    H = h * h * S
    k2 = stats.multivariate_normal(mean=np.zeros(d), cov=2 * H)
    k1 = stats.multivariate_normal(mean=np.zeros(d), cov=H)
    v = np.array([x[:, i] - x[:, j] for i in range(n) for j in range(i + 1, n)])
    return 2.0 / n ** 2 * np.sum(k2.pdf(v) - 2 * k1.pdf(v)) + k2.pdf(np.zeros(d)) / n


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_lscv_matches_library_densities(d):
    x = datagen.correlated_mixture(30, d, seed=40 + d).astype(np.float64)
    h = np.array([0.1, 0.4, 1.0, 2.5])
    g = oracle.lscv_h(x, h)["g"]
    for k in range(h.size):
        assert g[k] == pytest.approx(_lscv_mvn_bruteforce(x, h[k]), rel=1e-10, abs=1e-14)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_lscv_limits(d):
    x = datagen.correlated_mixture(50, d, seed=60 + d).astype(np.float64)
    n = x.shape[1]
    _, S = oracle.mean_cov(x)
    A = (4 * math.pi) ** (-d / 2) / math.sqrt(np.linalg.det(S))
    big, small = 1e7, 1e-7
    r = oracle.lscv_h(x, np.array([small, big]))
    g_small = r["g"][0] * small ** d / A
    g_big = r["g"][1] * big ** d / A
    assert g_small == pytest.approx(1.0 / n, rel=1e-12)
    assert g_big == pytest.approx((n - 1) / n * (1 - 2 ** (1 + d / 2)) + 1.0 / n, rel=1e-6)


def test_lscv_h_equals_lscv_H_at_scaled_covariance():
    for d in (1, 2, 3):
        x = datagen.correlated_mixture(60, d, seed=80 + d).astype(np.float64)
        _, S = oracle.mean_cov(x)
        h = np.array([0.3, 0.8])
        g = oracle.lscv_h(x, h)["g"]
        for k in range(2):
            assert oracle.lscv_H(x, h[k] ** 2 * S) == pytest.approx(g[k], rel=1e-12)


def test_lscv_H_general_matrix_vs_library():
    x = datagen.correlated_mixture(25, 2, seed=91).astype(np.float64)
    H = np.array([[0.4, 0.1], [0.1, 0.9]])
    n = x.shape[1]
    k2 = stats.multivariate_normal(mean=np.zeros(2), cov=2 * H)
    k1 = stats.multivariate_normal(mean=np.zeros(2), cov=H)
    v = np.array([x[:, i] - x[:, j] for i in range(n) for j in range(i + 1, n)])
    expect = 2.0 / n ** 2 * np.sum(k2.pdf(v) - 2 * k1.pdf(v)) + k2.pdf(np.zeros(2)) / n
    assert oracle.lscv_H(x, H) == pytest.approx(expect, rel=1e-11)


def test_lscv_invariances_and_argmin():
    x = datagen.correlated_mixture(120, 2, seed=5).astype(np.float64)
    h = oracle.grid_default(120, 2, 24)
    base = oracle.lscv_h(x, h)
    rng = datagen.rng(3)
    perm = oracle.lscv_h(x[:, rng.permutation(120)], h)
    assert np.allclose(perm["g"], base["g"], rtol=1e-12)
    shift = oracle.lscv_h(x + np.array([[5.0], [-2.0]]), h)
    assert np.allclose(shift["g"], base["g"], rtol=1e-9)
    M = np.array([[2.0, 0.5], [-0.3, 1.5]])
    aff = oracle.lscv_h(M @ x, h)
    assert np.allclose(aff["g"], base["g"] / abs(np.linalg.det(M)), rtol=1e-9)
    assert aff["argmin"] == base["argmin"]
    assert base["argmin"] == int(np.argmin(base["g"]))


def test_lscv_argmin_first_on_ties():
    x = datagen.mixture_1d(40, seed=2)
    h = np.array([0.5, 0.3, 0.3, 0.3, 0.9])
    r = oracle.lscv_h(x, h)
    assert r["g"][1] == r["g"][2] == r["g"][3]
    if r["argmin"] in (1, 2, 3):
        assert r["argmin"] == 1


def test_lscv_exp_sums_relation():
    # T = A (e - 2^(1+d/2) e^2) with e = exp(-S(v)/(4h^2)): the two separately
    # evaluated exponential sums reproduce the T sum.
    for d in (1, 3):
        x = datagen.correlated_mixture(70, d, seed=13).astype(np.float64)
        h = np.array([0.2, 0.7])
        skk, sk, st = oracle.lscv_sums(x, h)
        _, S = oracle.mean_cov(x)
        A = (4 * math.pi) ** (-d / 2) / math.sqrt(np.linalg.det(S))
        assert np.allclose(st, A * (skk - 2 ** (1 + d / 2) * sk), rtol=1e-12)


@pytest.mark.parametrize("d,n_h", [(1, 64), (2, 128), (3, 16)])
def test_octave_grid_sum_identity(d, n_h):
    """On the default grid (n_h/8 points per octave of 1/h^2: c_(k-P) = 2 c_k,
    reading R6), the K-term sum at bandwidth k is the K*K-term sum at k - P:
    exp(-S(v)/(2 h_k^2)) = exp(-S(v)/(4 h_(k-P)^2)) for every pair.  This is the
    identity the octave kernel uses (S2(k) = S1(k - P)); here it is checked on
    the oracle's separately evaluated sums."""
    n = 300
    x = datagen.correlated_mixture(n, d, seed=61 + d).astype(np.float64)
    h = oracle.grid_default(n, d, n_h)
    P = n_h // 8
    ref = oracle.lscv_h(x, h)
    assert np.allclose(ref["s_k"][P:], ref["s_kk"][:-P], rtol=1e-11, atol=0)


def test_lscv_block_decomposition_adds_up():
    x = datagen.correlated_mixture(90, 2, seed=17).astype(np.float64)
    h = np.array([0.25, 0.9])
    full = oracle.lscv_sums(x, h)
    cuts = [0, 30, 61, 90]
    acc = [np.zeros(2) for _ in range(3)]
    for a in range(3):
        for b in range(a, 3):
            part = oracle.lscv_sums(x, h, block=(cuts[a], cuts[a + 1], cuts[b], cuts[b + 1]))
            for k in range(3):
                acc[k] += part[k]
    for k in range(3):
        assert np.allclose(acc[k], full[k], rtol=1e-12)


def test_thread_count_does_not_change_results():
    if oracle.openmp_threads() < 2:
        pytest.skip("oracle built without OpenMP")
    x = datagen.skewed_column(300, seed=8)[0].astype(np.float64)
    h = np.array([0.1, 0.5])
    a = oracle.lscv_sums(x, h, threads=1)
    b = oracle.lscv_sums(x, h, threads=4)
    for k in range(3):
        assert np.array_equal(a[k], b[k])
    assert oracle.psi_pair_sum(x, 6, 3.0, threads=1) == oracle.psi_pair_sum(x, 6, 3.0, threads=3)


def test_toy8_regression_fixture():
    """The paper's 8-point toy set: values recorded from the oracle by
    tests/golden/make_golden.py (a regression fixture, not a paper pin)."""
    ref = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "toy8_oracle.json")))
    x = np.array(GOLD["toy_dataset"]["x"], dtype=np.float64)
    r = oracle.lscv_h(x, np.array(ref["h"]))
    assert np.allclose(r["g"], ref["g"], rtol=1e-13)
    assert r["argmin"] == ref["argmin"]
    p = oracle.plugin(x)
    for k in ("sigma", "g1", "psi6", "g2", "psi4", "h"):
        assert p[k] == pytest.approx(ref["plugin"][k], rel=1e-13)


# ------------------------------------------- exact leave-one-out, search

def _lscv_loo_d1_by_quadrature(x, h):
    """g_loo(h) = int fhat^2 - (2/n) sum_i fhat_{-i}(X_i), the integral by
    quadrature, the leave-one-out sum by library normal densities."""
    x = np.asarray(x, dtype=np.float64).ravel()
    n = x.size
    bw = h * np.std(x, ddof=1)
    fhat = lambda t: np.sum(stats.norm.pdf(t, loc=x, scale=bw)) / n
    pts = np.sort(x)
    val, _ = integrate.quad(lambda t: fhat(t) ** 2, pts[0] - 12 * bw, pts[-1] + 12 * bw, points=pts,
                            limit=2000, epsabs=0, epsrel=1e-12)
    loo = 0.0
    for i in range(n):
        loo += (np.sum(stats.norm.pdf(x[i] - x, scale=bw)) - stats.norm.pdf(0.0, scale=bw)) / (n - 1)
    return val - 2.0 * loo / n


def test_lscv_loo_matches_quadrature():
    x = datagen.mixture_1d(11, seed=4)[0]
    h = np.array([0.08, 0.3, 0.9])
    g = oracle.lscv_h_loo(x, h)
    for k in range(h.size):
        assert g[k] == pytest.approx(_lscv_loo_d1_by_quadrature(x, h[k]), rel=1e-8, abs=1e-12)


def test_lscv_loo_multivariate_library_densities():
    x = datagen.correlated_mixture(25, 3, seed=8).astype(np.float64)
    d, n = x.shape
    S = np.cov(x)
    for hh in (0.3, 1.1):
        H = hh * hh * S
        k2 = stats.multivariate_normal(mean=np.zeros(d), cov=2 * H)
        k1 = stats.multivariate_normal(mean=np.zeros(d), cov=H)
        v = np.array([x[:, i] - x[:, j] for i in range(n) for j in range(i + 1, n)])
        expect = (n * k2.pdf(np.zeros(d)) + 2 * np.sum(k2.pdf(v))) / n ** 2 - \
            4.0 / (n * (n - 1)) * np.sum(k1.pdf(v))
        assert oracle.lscv_h_loo(x, [hh])[0] == pytest.approx(expect, rel=1e-10)


def test_search_finds_the_dense_grid_minimum_of_a_unimodal_objective():
    x = datagen.rng(12).normal(0.0, 1.0, 400)
    z = oracle.h0(400, 1)
    a, b = z / 4, 4 * z
    dense = oracle.grid_log(a, b, 3000)
    gd = oracle.lscv_h(x, dense)["g"]
    hs, gs, rounds = oracle.lscv_search(x, a, b, P=8, rel_tol=1e-4)
    k = int(np.argmin(gd))
    step = dense[1] / dense[0]
    assert dense[k] / step ** 2 <= hs <= dense[k] * step ** 2
    assert gs <= gd[k] + 1e-12 * abs(gd[k])
    # each round keeps 2/(P+1) of the log-width
    expect = int(np.ceil(np.log(np.log(b / a) / 2e-4) / np.log(9 / 2)))
    assert rounds == expect


def test_search_loo_flag_uses_the_loo_objective():
    x = datagen.mixture_1d(300, seed=6)[0]
    z = oracle.h0(300, 1)
    h1, g1, _ = oracle.lscv_search(x, z / 4, 4 * z, loo=True)
    assert g1 == pytest.approx(oracle.lscv_h_loo(x, [h1])[0], rel=1e-14)
    h2, g2, _ = oracle.lscv_search(x, z / 4, 4 * z, loo=False)
    assert g2 == pytest.approx(oracle.lscv_h(x, [h2])["g"][0], rel=1e-14)


# ------------------------------------------- density evaluation and AQP

@pytest.mark.parametrize("d", [1, 2, 4])
def test_kde_eval_matches_library_densities(d):
    x = datagen.correlated_mixture(60, d, seed=120 + d).astype(np.float64)
    rng = datagen.rng(d)
    A = rng.normal(size=(d, d)) * 0.4
    H = A @ A.T + 0.3 * np.eye(d)
    q = rng.normal(size=(d, 9)) * 2
    f = oracle.kde_eval(x, H, q)
    mvn = stats.multivariate_normal(mean=np.zeros(d), cov=H)
    for k in range(q.shape[1]):
        expect = np.mean([mvn.pdf(q[:, k] - x[:, i]) for i in range(x.shape[1])])
        assert f[k] == pytest.approx(expect, rel=1e-11)


def test_kde_eval_integrates_to_one():
    x = datagen.mixture_1d(40, seed=3)
    H = np.array([[0.09]])
    val, _ = integrate.quad(lambda t: oracle.kde_eval(x, H, np.array([[t]]))[0], -20, 20, limit=400)
    assert val == pytest.approx(1.0, rel=1e-9)


def test_aqp_count_and_sum_match_quadrature():
    x = datagen.mixture_1d(30, seed=5)[0]
    n, h = x.size, 0.4
    lo = np.array([-3.0, -0.5, 1.0])
    hi = np.array([-1.0, 2.5, 1.2])
    c, s = oracle.aqp(x, h, lo, hi)
    fh = lambda t: np.sum(stats.norm.pdf(t, loc=x, scale=h)) / n
    for k in range(3):
        ce, _ = integrate.quad(lambda t: n * fh(t), lo[k], hi[k], epsabs=0, epsrel=1e-12, limit=200)
        se, _ = integrate.quad(lambda t: n * t * fh(t), lo[k], hi[k], epsabs=0, epsrel=1e-12, limit=200)
        assert c[k] == pytest.approx(ce, rel=1e-9)
        assert s[k] == pytest.approx(se, rel=1e-9, abs=1e-12)
    call, sall = oracle.aqp(x, h, [-1e3], [1e3])
    assert call[0] == pytest.approx(n, rel=1e-14)
    assert sall[0] == pytest.approx(np.sum(x), rel=1e-12)
