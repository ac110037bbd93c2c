"""FP64 CPU oracle for exact KDE bandwidth selection (arXiv 1505.01998).

TEST INFRASTRUCTURE ONLY.  The functions here wrap ``kde_oracle.c``, a plain,
slow, obviously correct C statement of the method (Sec. 4.4: PLUGIN, LSCV_h,
LSCV_H).  Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  It shares no code with the CUDA
library in ``paper_1505_01998_gb300`` and never imports it.

Samples are passed as a ``(d, n)`` float64 array (one sample per column, the
paper's d x n input matrix of Sec. 4.4.2) or a 1-D array for d = 1.

Every function's numerics are pinned by ``tests/test_oracle_*.py`` (closed
forms, brute force, quadrature, invariants); no function is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kde_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libkde_oracle.so")
_lock = threading.Lock()
_lib = None

OK, EDEGENERATE, EINVAL, ENOMEM = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available).

    ``-ffp-contract=off`` keeps every multiply and add separately rounded, so
    the oracle gives the same bits on x86-64 and AArch64.
    """
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", _SRC, "-o", _LIB_PATH + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        D, L, I, P = ctypes.c_double, ctypes.c_long, ctypes.c_int, ctypes.c_void_p
        sig = {
            "kdeo_have_openmp": (I, []),
            "kdeo_mean_cov": (I, [P, L, I, P, P]),
            "kdeo_invert": (I, [P, I, P, P]),
            "kdeo_hermite": (D, [I, D]),
            "kdeo_gauss_deriv": (D, [I, D]),
            "kdeo_psi_pair_sum_block": (D, [P, L, I, D, L, L, L, L, I]),
            "kdeo_psi_pair_sum": (D, [P, L, I, D, I]),
            "kdeo_psi_abs_pair_sum_block": (D, [P, L, I, D, L, L, L, L, I]),
            "kdeo_psi": (D, [P, L, I, D, I]),
            "kdeo_psi8_ns": (D, [D]),
            "kdeo_plugin_g1": (D, [D, L]),
            "kdeo_plugin_g2": (D, [D, L]),
            "kdeo_plugin_h": (D, [D, L]),
            "kdeo_plugin": (I, [P, L, I, P]),
            "kdeo_h0": (D, [L, I]),
            "kdeo_grid_log": (None, [D, D, I, P]),
            "kdeo_grid_default": (None, [L, I, I, P]),
            "kdeo_lscv_sums_block": (I, [P, L, I, P, I, L, L, L, L, P, P, P, I]),
            "kdeo_lscv_h": (I, [P, L, I, P, I, P, P, P, P, I]),
            "kdeo_lscv_H": (I, [P, L, I, P, P, I]),
            "kdeo_lscv_h_loo": (I, [P, L, I, P, I, P, I]),
            "kdeo_kde_eval": (I, [P, L, I, P, P, L, P, I]),
            "kdeo_aqp": (I, [P, L, D, P, P, L, P, P, I]),
            "kdeo_lscv_search": (I, [P, L, I, D, D, I, D, I, I, P, P, P, I]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


class PluginResult(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("var", "sigma", "psi8_ns", "g1", "psi6", "g2", "psi4", "h")] + [
                    ("status", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _as2d(x) -> np.ndarray:
    a = np.asarray(x, dtype=np.float64)
    if a.ndim == 1:
        a = a[None, :]
    return np.ascontiguousarray(a)


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def openmp_threads() -> int:
    """Threads the oracle would use by default (0 when built without OpenMP)."""
    return _load().kdeo_have_openmp()


def mean_cov(x):
    a = _as2d(x)
    d, n = a.shape
    mean = np.zeros(d)
    cov = np.zeros((d, d))
    rc = _load().kdeo_mean_cov(_p(a), n, d, _p(mean), _p(cov))
    if rc:
        raise ValueError(f"oracle mean_cov status {rc}")
    return mean, cov


def invert(A):
    A = np.ascontiguousarray(A, dtype=np.float64)
    d = A.shape[0]
    out = np.zeros_like(A)
    det = np.zeros(1)
    rc = _load().kdeo_invert(_p(A), d, _p(out), _p(det))
    return out, float(det[0]), rc


def hermite(r: int, x: float) -> float:
    return _load().kdeo_hermite(r, float(x))


def gauss_deriv(r: int, x: float) -> float:
    return _load().kdeo_gauss_deriv(r, float(x))


def psi_pair_sum(x, r: int, g: float, threads: int = 0, block=None) -> float:
    """sum over i<j of K^(r)((x_i - x_j)/g); ``block`` = (i0, i1, j0, j1)."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel())
    n = a.size
    if block is None:
        return _load().kdeo_psi_pair_sum(_p(a), n, r, float(g), threads)
    i0, i1, j0, j1 = (int(v) for v in block)
    return _load().kdeo_psi_pair_sum_block(_p(a), n, r, float(g), i0, i1, j0, j1, threads)


def psi_abs_pair_sum(x, r: int, g: float, threads: int = 0, block=None) -> float:
    """sum over i<j of |K^(r)((x_i - x_j)/g)| (magnitude scale for error statements)."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel())
    n = a.size
    i0, i1, j0, j1 = (0, n, 0, n) if block is None else (int(v) for v in block)
    return _load().kdeo_psi_abs_pair_sum_block(_p(a), n, r, float(g), i0, i1, j0, j1, threads)


def psi(x, r: int, g: float, threads: int = 0) -> float:
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel())
    return _load().kdeo_psi(_p(a), a.size, r, float(g), threads)


def psi8_ns(sigma: float) -> float:
    return _load().kdeo_psi8_ns(float(sigma))


def plugin_g1(psi8: float, n: int) -> float:
    return _load().kdeo_plugin_g1(float(psi8), int(n))


def plugin_g2(psi6: float, n: int) -> float:
    return _load().kdeo_plugin_g2(float(psi6), int(n))


def plugin_h(psi4: float, n: int) -> float:
    return _load().kdeo_plugin_h(float(psi4), int(n))


def plugin(x, threads: int = 0) -> dict:
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel())
    out = PluginResult()
    _load().kdeo_plugin(_p(a), a.size, threads, ctypes.byref(out))
    return out.as_dict()


def h0(n: int, d: int) -> float:
    return _load().kdeo_h0(int(n), int(d))


def grid_log(hmin: float, hmax: float, n_h: int) -> np.ndarray:
    out = np.zeros(n_h)
    _load().kdeo_grid_log(float(hmin), float(hmax), int(n_h), _p(out))
    return out


def grid_default(n: int, d: int, n_h: int) -> np.ndarray:
    """Log-spaced grid over Z(h0) = [h0/4, 4 h0) (Eq. LSCV-Zh0):
    h_k = (h0/4) 16^(k/n_h), k = 0 .. n_h-1."""
    out = np.zeros(n_h)
    _load().kdeo_grid_default(int(n), int(d), int(n_h), _p(out))
    return out


def lscv_sums(x, h, block=None, threads: int = 0):
    """(s_kk, s_k, s_t) pair sums of the LSCV_h objective over a pair block."""
    a = _as2d(x)
    d, n = a.shape
    hh = np.ascontiguousarray(np.asarray(h, dtype=np.float64).ravel())
    skk, sk, st = (np.zeros(hh.size) for _ in range(3))
    i0, i1, j0, j1 = (0, n, 0, n) if block is None else (int(v) for v in block)
    rc = _load().kdeo_lscv_sums_block(_p(a), n, d, _p(hh), hh.size, i0, i1, j0, j1,
                                      _p(skk), _p(sk), _p(st), threads)
    if rc:
        raise ValueError(f"oracle lscv_sums status {rc}")
    return skk, sk, st


def lscv_h(x, h, threads: int = 0):
    """g(h) on the grid, the argmin index, and the two exponential sums."""
    a = _as2d(x)
    d, n = a.shape
    hh = np.ascontiguousarray(np.asarray(h, dtype=np.float64).ravel())
    g, skk, sk = (np.zeros(hh.size) for _ in range(3))
    am = ctypes.c_int(0)
    rc = _load().kdeo_lscv_h(_p(a), n, d, _p(hh), hh.size, _p(g), ctypes.byref(am),
                             _p(skk), _p(sk), threads)
    if rc:
        raise ValueError(f"oracle lscv_h status {rc}")
    return {"g": g, "argmin": am.value, "s_kk": skk, "s_k": sk}


def lscv_h_loo(x, h, threads: int = 0) -> np.ndarray:
    """Exact leave-one-out g(h) on the grid."""
    a = _as2d(x)
    d, n = a.shape
    hh = np.ascontiguousarray(np.asarray(h, dtype=np.float64).ravel())
    g = np.zeros(hh.size)
    rc = _load().kdeo_lscv_h_loo(_p(a), n, d, _p(hh), hh.size, _p(g), threads)
    if rc:
        raise ValueError(f"oracle lscv_h_loo status {rc}")
    return g


def lscv_search(x, a: float, b: float, P: int = 8, rel_tol: float = 1e-4, max_rounds: int = 30,
                loo: bool = False, threads: int = 0):
    """Bracketing search for argmin g(h) over [a, b]: (h, g, rounds)."""
    arr = _as2d(x)
    d, n = arr.shape
    hb, gb = np.zeros(1), np.zeros(1)
    rounds = ctypes.c_int(0)
    rc = _load().kdeo_lscv_search(_p(arr), n, d, float(a), float(b), int(P), float(rel_tol),
                                  int(max_rounds), int(bool(loo)), _p(hb), _p(gb),
                                  ctypes.byref(rounds), threads)
    if rc:
        raise ValueError(f"oracle lscv_search status {rc}")
    return float(hb[0]), float(gb[0]), rounds.value


def kde_eval(x, H, q, threads: int = 0) -> np.ndarray:
    """fhat at the points q (d, m) with bandwidth matrix H."""
    a = _as2d(x)
    d, n = a.shape
    qq = np.ascontiguousarray(np.asarray(q, dtype=np.float64).reshape(d, -1))
    HH = np.ascontiguousarray(np.asarray(H, dtype=np.float64).reshape(d, d))
    f = np.zeros(qq.shape[1])
    rc = _load().kdeo_kde_eval(_p(a), n, d, _p(HH), _p(qq), qq.shape[1], _p(f), threads)
    if rc:
        raise ValueError(f"oracle kde_eval status {rc}")
    return f


def aqp(x, h: float, lo, hi, threads: int = 0):
    """(count, sum) over the ranges [lo_k, hi_k] of a univariate column."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel())
    l = np.ascontiguousarray(np.asarray(lo, dtype=np.float64).ravel())
    u = np.ascontiguousarray(np.asarray(hi, dtype=np.float64).ravel())
    c, s = np.zeros(l.size), np.zeros(l.size)
    _load().kdeo_aqp(_p(a), a.size, float(h), _p(l), _p(u), l.size, _p(c), _p(s), threads)
    return c, s


def lscv_H(x, H, threads: int = 0) -> float:
    a = _as2d(x)
    d, n = a.shape
    HH = np.ascontiguousarray(np.asarray(H, dtype=np.float64).reshape(d, d))
    g = np.zeros(1)
    rc = _load().kdeo_lscv_H(_p(a), n, d, _p(HH), _p(g), threads)
    if rc:
        raise ValueError(f"oracle lscv_H status {rc}")
    return float(g[0])
