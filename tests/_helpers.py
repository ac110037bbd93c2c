"""Shared helpers of the test suite: library access and the error metrics.

Error metrics (tolerance 1e-5, the stated FP32-path accuracy target):
  * LSCV exponential sums S1 = sum e, S2 = sum e^2 (positive terms): relative
    error |dS| / S.
  * g(h) changes sign over a grid, so its error is stated relative to
    max(|g|, scale) with scale = A h^-d (2 n^-2 (S1 + 2^(1+d/2) S2) + 1/n), the
    same expression with every term taken positive.
  * psi sums are signed: error relative to max(|sum|, sum |terms|).
  * A selected bandwidth that is not a grid point (the plug-in h) against
    the oracle's: |dh| / h <= H_TOL = 1e-4, the stated target for selected
    bandwidths.  h = (R(K) / (psi_4 n))^(1/5) carries a fifth of psi_4's
    error relative to psi_4 itself, which is its error relative to the
    magnitude scale times the cancellation ratio sum|terms| / |sum| (up to
    about 400 in the lognormal and mixture datasets of the batch workload).
"""
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

TOL = 1e-5
H_TOL = 1e-4


def built_lib():
    from paper_1505_01998_gb300 import build as B
    B.build()
    from paper_1505_01998_gb300 import gbkde
    gbkde.lib()
    return gbkde


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


def s_err(got, ref, npairs):
    """Error of a sum of positive exponentials.  Terms below 2^-126 are flushed
    to zero by the FP32 path (ex2.approx.ftz), so the error is relative to the
    sum, floored at the largest mass those terms can hold (npairs * 2^-126)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return np.abs(got - ref) / np.maximum(ref, npairs * 2.0 ** -126)


def g_scale(s1, s2, h, n, d, A):
    h = np.asarray(h, dtype=np.float64)
    return A * h ** (-d) * (2.0 / n ** 2 * (np.asarray(s1) + 2 ** (1 + d / 2) * np.asarray(s2)) + 1.0 / n)


def g_err(g_gpu, g_ref, s1, s2, h, n, d, A):
    scale = np.maximum(np.abs(g_ref), g_scale(s1, s2, h, n, d, A))
    return np.abs(np.asarray(g_gpu) - np.asarray(g_ref)) / scale


def lscv_A(x):
    import oracle
    _, S = oracle.mean_cov(x)
    d = S.shape[0]
    return (4 * math.pi) ** (-d / 2) / math.sqrt(np.linalg.det(S))


def argmin_ok(k_gpu, g_ref, tol_abs):
    """Same index, or a near tie: the oracle's g at the GPU index is within
    tol_abs of the oracle minimum."""
    k_ref = int(np.argmin(g_ref))
    return k_gpu == k_ref or (g_ref[k_gpu] - g_ref[k_ref]) <= tol_abs
