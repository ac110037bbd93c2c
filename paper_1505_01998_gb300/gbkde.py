"""Thin Python binding of libgbkde (include/gbkde.h).

Argument marshalling only: every step of the method runs in the CUDA library.
PyTorch provides device memory (the workspace and device-resident samples) and
CUDA streams.  Functions keep the C names; structs mirror the C structs.
If the shared library has not been built, every call raises: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgbkde.so")

KDE_OK, KDE_EINVAL, KDE_ENOMEM, KDE_ECUDA, KDE_EDEGENERATE = 0, 1, 2, 3, 4
KDE_EBUSY, KDE_EAGAIN, KDE_ETIMEDOUT, KDE_ECANCELLED, KDE_ENOTFOUND, KDE_EINTERNAL = 5, 6, 7, 8, 9, 10
KDE_F32, KDE_F64 = 0, 1
KDE_FP32_KAHAN, KDE_FP32_PLAIN = 0, 1
KDE_GRID_DEFAULT_Z, KDE_GRID_EXPLICIT, KDE_GRID_LOG = 0, 1, 2
KDE_METHOD_LSCV, KDE_METHOD_PLUGIN = 1, 2
KDE_FLAG_MIN_AT_LOWER_EDGE, KDE_FLAG_MIN_AT_UPPER_EDGE = 1, 2
KDE_MAX_D, KDE_MAX_NH = 16, 1024


class KdeError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"[status {status}] {msg}")
        self.status = status


class kde_grid(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n_h", ctypes.c_int),
                ("h", ctypes.POINTER(ctypes.c_double)),
                ("h_min", ctypes.c_double), ("h_max", ctypes.c_double)]


class kde_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("tile", ctypes.c_int),
                ("bw_per_thread", ctypes.c_int), ("tiles_per_item", ctypes.c_int),
                ("ctas_per_sm", ctypes.c_int), ("cv", ctypes.c_int)]


KDE_CV_PAPER, KDE_CV_LOO = 0, 1


class kde_result(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int) for k in ("status", "method", "argmin", "flags", "n_h", "d")] + [
        (k, ctypes.c_double) for k in ("h", "h_data", "g_min", "sigma", "psi8_ns", "g1", "psi6",
                                       "g2", "psi4", "logdet_S", "h_plugin")]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class kde_request(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("dtype", ctypes.c_int), ("d", ctypes.c_int),
                ("n", ctypes.c_int64), ("methods", ctypes.c_int), ("grid", kde_grid)]


_lock = threading.Lock()
_lib = None

# C signatures: name -> (restype, argtypes)
_P, _I, _L, _D, _S = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
_DP = ctypes.POINTER(ctypes.c_double)
SIGNATURES = {
    "kde_version": (ctypes.c_char_p, []),
    "kde_last_error": (_I, [ctypes.c_char_p, _S]),
    "kde_status_string": (ctypes.c_char_p, [_I]),
    "kde_tile_count": (_I, [_L, _I, ctypes.POINTER(ctypes.c_int64)]),
    "kde_tile_coords": (_I, [_L, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "kde_default_grid": (_I, [_L, _I, _I, _DP]),
    "kde_workspace_size": (_I, [_L, _I, _I, ctypes.POINTER(kde_opts), ctypes.POINTER(ctypes.c_size_t)]),
    "kde_ws_result_offset": (_I, [ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
    "kde_lscv": (_I, [_P, _I, _L, _I, ctypes.POINTER(kde_grid), ctypes.POINTER(kde_opts), _P, _S, _P,
                      _DP, _DP, ctypes.POINTER(kde_result)]),
    "kde_lscv_async": (_I, [_P, _I, _L, _I, ctypes.POINTER(kde_grid), ctypes.POINTER(kde_opts), _P,
                            _S, _P]),
    "kde_lscv_host": (_I, [_P, _I, _L, _I, ctypes.POINTER(kde_grid), ctypes.POINTER(kde_opts), _P, _S,
                           _P, _DP, ctypes.POINTER(kde_result)]),
    "kde_lscv_tile_sums": (_I, [_P, _I, _L, _I, _DP, _I, _L, _L, ctypes.POINTER(kde_opts), _P, _S, _P,
                                _DP, _DP]),
    "kde_plugin": (_I, [_P, _I, _L, ctypes.POINTER(kde_opts), _P, _S, _P, ctypes.POINTER(kde_result)]),
    "kde_plugin_async": (_I, [_P, _I, _L, ctypes.POINTER(kde_opts), _P, _S, _P]),
    "kde_plugin_host": (_I, [_P, _I, _L, ctypes.POINTER(kde_opts), _P, _S, _P,
                             ctypes.POINTER(kde_result)]),
    "kde_set_kernel_events": (_I, [_P, _P, _P, _P]),
    "kde_psi_tile_sums": (_I, [_P, _I, _L, _I, _D, _L, _L, ctypes.POINTER(kde_opts), _P, _S, _P, _DP]),
    "kde_psi_tile_edge": (_I, [_L, ctypes.POINTER(kde_opts), ctypes.POINTER(ctypes.c_int)]),
    "kde_probe_alu": (_I, [_P, _S, _P, _DP, _DP, _DP, _DP, ctypes.POINTER(ctypes.c_int), _DP]),
    "kde_lscv_H_workspace_size": (_I, [_L, _I, _I, ctypes.POINTER(kde_opts), ctypes.POINTER(_S)]),
    "kde_lscv_H": (_I, [_P, _I, _L, _I, _DP, _I, ctypes.POINTER(kde_opts), _P, _S, _P, _DP]),
    "kde_batch_plan_create": (_I, [ctypes.POINTER(kde_request), _I, ctypes.POINTER(kde_opts),
                                   ctypes.POINTER(_P), ctypes.POINTER(_S)]),
    "kde_batch_run_async": (_I, [_P, _P, _S, _P]),
    "kde_batch_run": (_I, [_P, _P, _S, _P, ctypes.POINTER(kde_result)]),
    "kde_batch_results": (_I, [_P, ctypes.POINTER(kde_result)]),
    "kde_batch_g": (_I, [_P, _P, _I, _DP]),
    "kde_batch_plan_destroy": (_I, [_P]),
    "kde_batch_workspace_size": (_I, [ctypes.POINTER(kde_request), _I, ctypes.POINTER(kde_opts),
                                      ctypes.POINTER(_S)]),
    "kde_select_batch": (_I, [ctypes.POINTER(kde_request), _I, ctypes.POINTER(kde_opts), _P, _S, _P,
                              ctypes.POINTER(kde_result)]),
    "kde_serve_create": (_I, [ctypes.c_void_p, ctypes.POINTER(_P)]),
    "kde_serve_submit": (_I, [_P, ctypes.POINTER(kde_request), ctypes.POINTER(ctypes.c_uint64)]),
    "kde_serve_poll": (_I, [_P, ctypes.c_uint64, ctypes.POINTER(kde_result)]),
    "kde_serve_wait": (_I, [_P, ctypes.c_uint64, _I, ctypes.POINTER(kde_result)]),
    "kde_serve_cancel": (_I, [_P, ctypes.c_uint64]),
    "kde_serve_stats": (_I, [_P, ctypes.c_void_p]),
    "kde_serve_destroy": (_I, [_P]),
    "kde_lscv_noalloc": (_I, [_P, _I, _L, _I, ctypes.POINTER(kde_grid), ctypes.POINTER(kde_opts), _P,
                              _DP, _DP, ctypes.POINTER(kde_result)]),
    "kde_lscv_logdet": (_I, [_P, _I, _L, _I, _P, _S, _P, _DP]),
    "kde_autotune": (_I, [_P, _I, _L, _I, _I, _I, _P, _S, _P, ctypes.POINTER(kde_opts), _DP]),
    "kde_sample_covariance": (_I, [_P, _I, _L, _I, _P, _S, _P, _DP]),
    "kde_lscv_search": (_I, [_P, _I, _L, _I, _D, _D, _D, _I, ctypes.POINTER(kde_opts), _P, _S, _P,
                             ctypes.POINTER(kde_result), ctypes.POINTER(ctypes.c_int)]),
    "kde_lscv_H_minimize": (_I, [_P, _I, _L, _I, _DP, _I, _D, ctypes.POINTER(kde_opts), _P, _S, _P,
                                 _DP, _DP, ctypes.POINTER(ctypes.c_int)]),
    "kde_eval_workspace_size": (_I, [_L, _I, _L, ctypes.POINTER(ctypes.c_size_t)]),
    "kde_eval": (_I, [_P, _I, _L, _I, _DP, _P, _L, _P, _S, _P, _DP]),
    "kde_aqp_workspace_size": (_I, [_L, _I, ctypes.POINTER(ctypes.c_size_t)]),
    "kde_aqp": (_I, [_P, _I, _L, _D, _DP, _DP, _I, _P, _S, _P, _DP, _DP]),
    "kde_autotune_clear": (_I, []),
    "kde_autotune_save": (_I, [ctypes.c_char_p]),
    "kde_autotune_load": (_I, [ctypes.c_char_p]),
    "kde_lscv_merge": (_I, [_L, _I, _D, _DP, _I, _DP, _DP, _DP, ctypes.POINTER(kde_result)]),
    "kde_plugin_merge": (_I, [_L, _I, _D, ctypes.POINTER(kde_result)]),
    "kde_item_tiles": (_I, [_L, _I, _DP, _I, ctypes.POINTER(kde_opts), ctypes.POINTER(ctypes.c_int),
                            ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                            ctypes.POINTER(ctypes.c_int)]),
}


def kde_lscv_search(x, h_lo=0.0, h_hi=0.0, rel_tol=1e-4, max_rounds=30, opts=None, ws=None,
                    stream=None):
    """Bracketing search (8 points per round); returns (result dict, rounds)."""
    ptr, dt, n, d = _samples(x)
    if ws is None:
        ws = workspace(kde_workspace_size(n, d, 8, opts), x.device)
    wp, wn = _ws(ws)
    res = kde_result()
    rounds = ctypes.c_int(0)
    _check(lib().kde_lscv_search(ptr, dt, n, d, float(h_lo), float(h_hi), float(rel_tol),
                                 int(max_rounds), ctypes.byref(opts) if opts else None, wp, wn,
                                 _stream_handle(stream), ctypes.byref(res), ctypes.byref(rounds)))
    return res.as_dict(), rounds.value


def kde_sample_covariance(x, ws=None, stream=None) -> np.ndarray:
    ptr, dt, n, d = _samples(x)
    if ws is None:
        ws = workspace(kde_workspace_size(n, d, 1), x.device)
    wp, wn = _ws(ws)
    out = np.zeros(d * d)
    _check(lib().kde_sample_covariance(ptr, dt, n, d, wp, wn, _stream_handle(stream), _dp(out)))
    return out.reshape(d, d)


def kde_lscv_H_minimize(x, H_start=None, max_iter=200, ftol=1e-8, opts=None, ws=None, stream=None):
    """Nelder-Mead minimisation of g(H); returns (H, g, number of g evaluations)."""
    ptr, dt, n, d = _samples(x)
    if ws is None:
        p = d * (d + 1) // 2
        ws = workspace(max(kde_workspace_size(n, d, 1), kde_lscv_H_workspace_size(n, d, max(4, p + 1))),
                       x.device)
    wp, wn = _ws(ws)
    H0 = None
    if H_start is not None:
        H0 = np.ascontiguousarray(np.asarray(H_start, dtype=np.float64).reshape(d, d))
    H = np.zeros(d * d)
    g = np.zeros(1)
    ev = ctypes.c_int(0)
    _check(lib().kde_lscv_H_minimize(ptr, dt, n, d, _dp(H0) if H0 is not None else None, int(max_iter),
                                     float(ftol), ctypes.byref(opts) if opts else None, wp, wn,
                                     _stream_handle(stream), _dp(H), _dp(g), ctypes.byref(ev)))
    return H.reshape(d, d), float(g[0]), ev.value


KDE_TUNE_LATENCY, KDE_TUNE_THROUGHPUT = 0, 1


def kde_autotune(x, n_h: int, mode: int = KDE_TUNE_THROUGHPUT, ws=None, stream=None):
    """Tune the LSCV geometry on device samples x; returns (kde_opts, evals/s).
    The winner is cached and used by later calls that leave options at 0."""
    ptr, dt, n, d = _samples(x)
    if ws is None:
        ws = workspace(1 << 30, x.device)
    wp, wn = _ws(ws)
    best = kde_opts()
    rate = np.zeros(1)
    _check(lib().kde_autotune(ptr, dt, n, d, int(n_h), int(mode), wp, wn, _stream_handle(stream),
                              ctypes.byref(best), _dp(rate)))
    return best, float(rate[0])


def kde_autotune_clear():
    _check(lib().kde_autotune_clear())


def kde_autotune_save(path: str):
    _check(lib().kde_autotune_save(str(path).encode()))


def kde_autotune_load(path: str):
    _check(lib().kde_autotune_load(str(path).encode()))


def kde_lscv_logdet(x, ws=None, stream=None) -> float:
    ptr, dt, n, d = _samples(x)
    if ws is None:
        ws = workspace(kde_workspace_size(n, d, 1), x.device)
    wp, wn = _ws(ws)
    out = np.zeros(1)
    _check(lib().kde_lscv_logdet(ptr, dt, n, d, wp, wn, _stream_handle(stream), _dp(out)))
    return float(out[0])


def kde_lscv_merge(n: int, d: int, logdet_S: float, h, s1, s2):
    """g(h) and the argmin from summed shard sums (host FP64)."""
    hh, a, b = (np.ascontiguousarray(np.asarray(v, dtype=np.float64).ravel()) for v in (h, s1, s2))
    g = np.zeros(hh.size)
    res = kde_result()
    _check(lib().kde_lscv_merge(int(n), int(d), float(logdet_S), _dp(hh), hh.size, _dp(a), _dp(b),
                                _dp(g), ctypes.byref(res)))
    return res.as_dict(), g

def kde_plugin_merge(n: int, stage: int, value: float, res: dict | None = None) -> dict:
    """One host step of a sharded PLUGIN chain: stage 8 (value = sigma),
    6 (value = summed psi_6 pair sum at g1) or 4 (psi_4 pair sum at g2)."""
    r = kde_result()
    if res is not None:
        for k, _ in kde_result._fields_:
            setattr(r, k, res[k])
    _check(lib().kde_plugin_merge(int(n), int(stage), float(value), ctypes.byref(r)))
    return r.as_dict()


def kde_item_tiles(n: int, d: int, n_h: int, opts: kde_opts | None = None, h=None) -> dict:
    """Tile edges and tiles per item of the single-GPU geometry on the grid h
    (None: the default grid of n_h points)."""
    v = [ctypes.c_int(0) for _ in range(4)]
    hh = None if h is None else np.ascontiguousarray(np.asarray(h, dtype=np.float64).ravel())
    if hh is not None:
        n_h = hh.size
    _check(lib().kde_item_tiles(int(n), int(d), _dp(hh) if hh is not None else None, int(n_h),
                                ctypes.byref(opts) if opts else None, *(ctypes.byref(x) for x in v)))
    return {"lscv_tile": v[0].value, "lscv_K": v[1].value, "psi_tile": v[2].value, "psi_K": v[3].value}


KDE_NOALLOC_MAX_BYTES = 16 << 20


def kde_lscv_noalloc(x, grid, opts=None, stream=None):
    """LSCV_h selection using the library's built-in scratch buffer instead of
    a caller workspace (for callers that cannot allocate device memory).
    Returns (result dict, g, h)."""
    ptr, dt, n, d = _samples(x)
    g = np.zeros(grid.n_h)
    h = np.zeros(grid.n_h)
    res = kde_result()
    _check(lib().kde_lscv_noalloc(ptr, dt, n, d, ctypes.byref(grid),
                                  ctypes.byref(opts) if opts else None, _stream_handle(stream),
                                  _dp(g), _dp(h), ctypes.byref(res)))
    return res.as_dict(), g, h


def kde_eval_workspace_size(n: int, d: int, m: int) -> int:
    out = ctypes.c_size_t(0)
    _check(lib().kde_eval_workspace_size(n, d, m, ctypes.byref(out)))
    return out.value


def kde_eval(x, H, q, ws=None, stream=None) -> np.ndarray:
    """Density estimate with bandwidth matrix H (d x d, or a scalar h^2 for
    d = 1) at the device query points q (d, m), from device samples x (d, n)."""
    ptr, dt, n, d = _samples(x)
    qp, qdt, m, qd = _samples(q)
    if qd != d or qdt != dt:
        raise ValueError("queries must have the samples' dimension and dtype")
    Hm = np.ascontiguousarray(np.asarray(H, dtype=np.float64).reshape(d, d))
    if ws is None:
        ws = workspace(kde_eval_workspace_size(n, d, m), x.device)
    wp, wn = _ws(ws)
    f = np.zeros(m)
    _check(lib().kde_eval(ptr, dt, n, d, _dp(Hm), qp, m, wp, wn, _stream_handle(stream), _dp(f)))
    return f


def kde_aqp_workspace_size(n: int, m: int) -> int:
    out = ctypes.c_size_t(0)
    _check(lib().kde_aqp_workspace_size(n, m, ctypes.byref(out)))
    return out.value


def kde_aqp(x, h: float, lo, hi, ws=None, stream=None):
    """Approximate Count and Sum over the ranges [lo_k, hi_k] from device
    samples x (n,) and bandwidth h.  Returns (count, sum) arrays."""
    ptr, dt, n, d = _samples(x)
    if d != 1:
        raise ValueError("range aggregates take one column")
    a = np.ascontiguousarray(np.asarray(lo, dtype=np.float64).ravel())
    b = np.ascontiguousarray(np.asarray(hi, dtype=np.float64).ravel())
    if a.size != b.size:
        raise ValueError("lo and hi differ in length")
    m = a.size
    if ws is None:
        ws = workspace(kde_aqp_workspace_size(n, m), x.device)
    wp, wn = _ws(ws)
    cnt = np.zeros(m)
    sm = np.zeros(m)
    _check(lib().kde_aqp(ptr, dt, n, float(h), _dp(a), _dp(b), m, wp, wn, _stream_handle(stream),
                         _dp(cnt), _dp(sm)))
    return cnt, sm


class kde_serve_config(ctypes.Structure):
    _fields_ = [("arena", ctypes.c_void_p), ("arena_bytes", ctypes.c_size_t),
                ("max_slots", ctypes.c_int), ("max_queue", ctypes.c_int),
                ("quantum_evals", ctypes.c_double), ("step_deadline_ms", ctypes.c_int),
                ("device", ctypes.c_int), ("opts", ctypes.POINTER(kde_opts))]


class kde_serve_stats_t(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in ("submitted", "completed", "failed", "cancelled",
                                                "rejected")] + [
        (k, ctypes.c_double) for k in ("p50_ms", "p99_ms", "mean_ms", "max_ms", "p50_wait_ms",
                                       "p99_wait_ms", "requests_per_s", "evals_per_s")] + [
        ("steps", ctypes.c_int64), ("queue_depth_max", ctypes.c_int), ("active_max", ctypes.c_int),
        ("arena_peak_bytes", ctypes.c_size_t)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


def lib():
    """Load libgbkde.so (raises if it has not been built)."""
    global _lib
    L = _lib
    if L is not None:  # loaded: no lock on the per-call path
        return L
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def _check(rc: int):
    if rc != KDE_OK:
        buf = ctypes.create_string_buffer(512)
        lib().kde_last_error(buf, 512)
        raise KdeError(rc, buf.value.decode(errors="replace"))


def _dp(a: np.ndarray):
    # a ctypes array over the numpy buffer converts to double* at the call
    # (a third of the cost of ndarray.ctypes.data_as, a few us per call)
    if a.dtype == np.float64 and a.flags.c_contiguous and a.flags.writeable and a.size > 0:
        return (ctypes.c_double * a.size).from_buffer(a)
    return a.ctypes.data_as(_DP)


# ------------------------------------------------------------------ helpers

def make_opts(precision=KDE_FP32_KAHAN, tile=0, bw_per_thread=0, tiles_per_item=0, ctas_per_sm=0,
              cv=KDE_CV_PAPER):
    return kde_opts(precision, tile, bw_per_thread, tiles_per_item, ctas_per_sm, cv)


def make_grid(h=None, n_h=None, h_min=None, h_max=None):
    """Explicit grid from an array h, log grid from (h_min, h_max, n_h), or the
    default Z(h0) grid from n_h alone.  Returns (kde_grid, keepalive)."""
    if h is not None:
        arr = np.ascontiguousarray(np.asarray(h, dtype=np.float64).ravel())
        return kde_grid(KDE_GRID_EXPLICIT, arr.size, _dp(arr), 0.0, 0.0), arr
    if h_min is not None:
        return kde_grid(KDE_GRID_LOG, int(n_h), None, float(h_min), float(h_max)), None
    return kde_grid(KDE_GRID_DEFAULT_Z, int(n_h), None, 0.0, 0.0), None


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.float32:
        return KDE_F32
    if t.dtype == torch.float64:
        return KDE_F64
    raise TypeError(f"samples must be float32 or float64, got {t.dtype}")


def _samples(x):
    """(d, n) contiguous device tensor -> (ptr, dtype, n, d)."""
    if x.dim() == 1:
        x = x[None, :]
    if not x.is_cuda:
        raise ValueError("samples must be a CUDA tensor; use kde_lscv_host for host data")
    if not x.is_contiguous():
        raise ValueError("samples must be contiguous (d, n)")
    return ctypes.c_void_p(x.data_ptr()), _dtype_code(x), int(x.shape[1]), int(x.shape[0])


def kde_version() -> str:
    return lib().kde_version().decode()


def kde_tile_count(n: int, tile: int) -> int:
    out = ctypes.c_int64(0)
    _check(lib().kde_tile_count(int(n), int(tile), ctypes.byref(out)))
    return out.value


def kde_tile_coords(bx: int):
    l, q = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib().kde_tile_coords(int(bx), ctypes.byref(l), ctypes.byref(q)))
    return l.value, q.value


def kde_default_grid(n: int, d: int, n_h: int) -> np.ndarray:
    out = np.zeros(n_h)
    _check(lib().kde_default_grid(int(n), int(d), int(n_h), _dp(out)))
    return out


def kde_workspace_size(n: int, d: int, n_h: int, opts: kde_opts | None = None) -> int:
    out = ctypes.c_size_t(0)
    _check(lib().kde_workspace_size(int(n), int(d), int(n_h),
                                    ctypes.byref(opts) if opts else None, ctypes.byref(out)))
    return out.value


def kde_ws_result_offset():
    r, g = ctypes.c_size_t(0), ctypes.c_size_t(0)
    _check(lib().kde_ws_result_offset(ctypes.byref(r), ctypes.byref(g)))
    return r.value, g.value


def workspace(nbytes: int, device=None):
    """A device workspace (torch uint8 tensor, 256-byte aligned)."""
    import torch
    t = torch.empty(int(nbytes) + 256, dtype=torch.uint8, device=device or "cuda")
    off = (-t.data_ptr()) % 256
    return t[off:off + int(nbytes)]


def _ws(ws):
    return ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(ws.numel())


def kde_lscv(x, grid: kde_grid, opts: kde_opts | None = None, ws=None, stream=None):
    """LSCV_h selection on device samples x (d, n).  Returns (result dict, g, h)."""
    ptr, dt, n, d = _samples(x)
    if ws is None:
        ws = workspace(kde_workspace_size(n, d, grid.n_h, opts), x.device)
    wp, wn = _ws(ws)
    g = np.zeros(grid.n_h)
    h = np.zeros(grid.n_h)
    res = kde_result()
    _check(lib().kde_lscv(ptr, dt, n, d, ctypes.byref(grid), ctypes.byref(opts) if opts else None,
                          wp, wn, _stream_handle(stream), _dp(g), _dp(h), ctypes.byref(res)))
    return res.as_dict(), g, h


def kde_lscv_async(x, grid: kde_grid, opts: kde_opts | None, ws, stream=None):
    ptr, dt, n, d = _samples(x)
    wp, wn = _ws(ws)
    _check(lib().kde_lscv_async(ptr, dt, n, d, ctypes.byref(grid),
                                ctypes.byref(opts) if opts else None, wp, wn, _stream_handle(stream)))


def kde_lscv_host(x_host: np.ndarray, grid: kde_grid, opts: kde_opts | None, ws, stream=None):
    """LSCV_h selection on HOST samples (copied into the workspace on the stream)."""
    a = np.ascontiguousarray(x_host)
    if a.ndim == 1:
        a = a[None, :]
    dt = KDE_F64 if a.dtype == np.float64 else KDE_F32
    if a.dtype not in (np.float32, np.float64):
        raise TypeError("samples must be float32 or float64")
    wp, wn = _ws(ws)
    g = np.zeros(grid.n_h)
    res = kde_result()
    _check(lib().kde_lscv_host(ctypes.c_void_p(a.ctypes.data), dt, a.shape[1], a.shape[0],
                               ctypes.byref(grid), ctypes.byref(opts) if opts else None, wp, wn,
                               _stream_handle(stream), _dp(g), ctypes.byref(res)))
    return res.as_dict(), g


def kde_lscv_tile_sums(x, h, tile_begin: int, tile_end: int, opts: kde_opts | None = None,
                       ws=None, stream=None):
    ptr, dt, n, d = _samples(x)
    hh = np.ascontiguousarray(np.asarray(h, dtype=np.float64).ravel())
    if ws is None:
        ws = workspace(kde_workspace_size(n, d, hh.size, opts), x.device)
    wp, wn = _ws(ws)
    s1, s2 = np.zeros(hh.size), np.zeros(hh.size)
    _check(lib().kde_lscv_tile_sums(ptr, dt, n, d, _dp(hh), hh.size, int(tile_begin), int(tile_end),
                                    ctypes.byref(opts) if opts else None, wp, wn,
                                    _stream_handle(stream), _dp(s1), _dp(s2)))
    return s1, s2


def kde_plugin(x, opts: kde_opts | None = None, ws=None, stream=None) -> dict:
    ptr, dt, n, d = _samples(x)
    if d != 1:
        raise ValueError("PLUGIN is univariate")
    if ws is None:
        ws = workspace(kde_workspace_size(n, 1, 0, opts), x.device)
    wp, wn = _ws(ws)
    res = kde_result()
    _check(lib().kde_plugin(ptr, dt, n, ctypes.byref(opts) if opts else None, wp, wn,
                            _stream_handle(stream), ctypes.byref(res)))
    return res.as_dict()


def kde_plugin_async(x, opts: kde_opts | None, ws, stream=None):
    ptr, dt, n, d = _samples(x)
    wp, wn = _ws(ws)
    _check(lib().kde_plugin_async(ptr, dt, n, ctypes.byref(opts) if opts else None, wp, wn,
                                  _stream_handle(stream)))


def kde_plugin_host(x_host: np.ndarray, opts: kde_opts | None, ws, stream=None) -> dict:
    a = np.ascontiguousarray(x_host).ravel()
    if a.dtype not in (np.float32, np.float64):
        raise TypeError("samples must be float32 or float64")
    dt = KDE_F64 if a.dtype == np.float64 else KDE_F32
    wp, wn = _ws(ws)
    res = kde_result()
    _check(lib().kde_plugin_host(ctypes.c_void_p(a.ctypes.data), dt, a.size,
                                 ctypes.byref(opts) if opts else None, wp, wn,
                                 _stream_handle(stream), ctypes.byref(res)))
    return res.as_dict()


def kde_set_kernel_events(lscv_begin=None, lscv_end=None, psi_begin=None, psi_end=None):
    """torch.cuda.Event objects (or None) recorded around the pair kernels."""
    def h(e):
        return ctypes.c_void_p(e.cuda_event) if e is not None else None
    _check(lib().kde_set_kernel_events(h(lscv_begin), h(lscv_end), h(psi_begin), h(psi_end)))


def kde_psi_tile_edge(n: int, opts: kde_opts | None = None) -> int:
    t = ctypes.c_int(0)
    _check(lib().kde_psi_tile_edge(int(n), ctypes.byref(opts) if opts else None, ctypes.byref(t)))
    return t.value


def kde_psi_tile_sums(x, r: int, g: float, tile_begin: int, tile_end: int,
                      opts: kde_opts | None = None, ws=None, stream=None) -> float:
    ptr, dt, n, d = _samples(x)
    if ws is None:
        ws = workspace(kde_workspace_size(n, 1, 0, opts), x.device)
    wp, wn = _ws(ws)
    out = np.zeros(1)
    _check(lib().kde_psi_tile_sums(ptr, dt, n, int(r), float(g), int(tile_begin), int(tile_end),
                                   ctypes.byref(opts) if opts else None, wp, wn,
                                   _stream_handle(stream), _dp(out)))
    return float(out[0])


def kde_probe_alu(ws=None, stream=None) -> dict:
    if ws is None:
        ws = workspace(1 << 20)
    wp, wn = _ws(ws)
    m, f, f2, ma, mhz = (np.zeros(1) for _ in range(5))
    sms = ctypes.c_int(0)
    _check(lib().kde_probe_alu(wp, wn, _stream_handle(stream), _dp(m), _dp(f), _dp(f2), _dp(ma),
                               ctypes.byref(sms), _dp(mhz)))
    return {"mufu_ex2_per_clk_sm": float(m[0]), "ffma_lanes_per_clk_sm": float(f[0]),
            "ffma2_lanes_per_clk_sm": float(f2[0]), "fmul2_fadd2_lanes_per_clk_sm": float(ma[0]),
            "sm_count": sms.value, "sm_mhz": float(mhz[0])}


def read_ws_result(ws, n_h: int = 0):
    """Copy the result (and g[]) left in a workspace by an _async call."""
    import torch
    roff, goff = kde_ws_result_offset()
    raw = ws[roff:roff + ctypes.sizeof(kde_result)].cpu().numpy().tobytes()
    res = kde_result.from_buffer_copy(raw).as_dict()
    g = None
    if n_h:
        g = ws[goff:goff + 8 * n_h].cpu().view(torch.float64).numpy().copy()
    return res, g


# ------------------------------------------------------------------ LSCV_H

def kde_lscv_H_workspace_size(n: int, d: int, m: int, opts: kde_opts | None = None) -> int:
    out = ctypes.c_size_t(0)
    _check(lib().kde_lscv_H_workspace_size(int(n), int(d), int(m),
                                           ctypes.byref(opts) if opts else None, ctypes.byref(out)))
    return out.value


def kde_lscv_H(x, H, opts: kde_opts | None = None, ws=None, stream=None) -> np.ndarray:
    """g(H) for each of the m bandwidth matrices H (m, d, d) on device samples x (d, n)."""
    ptr, dt, n, d = _samples(x)
    HH = np.ascontiguousarray(np.asarray(H, dtype=np.float64).reshape(-1, d, d))
    m = HH.shape[0]
    if ws is None:
        ws = workspace(kde_lscv_H_workspace_size(n, d, m, opts), x.device)
    wp, wn = _ws(ws)
    g = np.zeros(m)
    _check(lib().kde_lscv_H(ptr, dt, n, d, _dp(HH), m, ctypes.byref(opts) if opts else None,
                            wp, wn, _stream_handle(stream), _dp(g)))
    return g


# ------------------------------------------------------------------ batches

def make_request(x, methods=KDE_METHOD_LSCV | KDE_METHOD_PLUGIN, grid: kde_grid | None = None):
    """A kde_request for device samples x (d, n) (or host numpy samples for the
    server).  Returns (request, keepalive)."""
    if isinstance(x, np.ndarray):
        a = np.ascontiguousarray(x if x.ndim == 2 else x[None, :])
        ptr, dt, n, d = a.ctypes.data, (KDE_F64 if a.dtype == np.float64 else KDE_F32), a.shape[1], a.shape[0]
        keep = a
    else:
        p, dt, n, d = _samples(x)
        ptr, keep = p.value, x
    g = grid if grid is not None else kde_grid(KDE_GRID_DEFAULT_Z, 128, None, 0.0, 0.0)
    return kde_request(ptr, dt, d, n, methods, g), keep


class BatchPlan:
    """Owner of a kde_batch_plan (destroyed with the object)."""

    def __init__(self, requests, opts: kde_opts | None = None, keepalive=()):
        self.n = len(requests)
        self._reqs = (kde_request * self.n)(*requests)
        self._keep = list(keepalive)
        self.opts = opts
        h = ctypes.c_void_p(0)
        nb = ctypes.c_size_t(0)
        _check(lib().kde_batch_plan_create(self._reqs, self.n, ctypes.byref(opts) if opts else None,
                                           ctypes.byref(h), ctypes.byref(nb)))
        self.handle = h
        self.ws_bytes = nb.value

    def run(self, ws, stream=None):
        wp, wn = _ws(ws)
        out = (kde_result * self.n)()
        _check(lib().kde_batch_run(self.handle, wp, wn, _stream_handle(stream), out))
        return [r.as_dict() for r in out]

    def run_async(self, ws, stream=None):
        wp, wn = _ws(ws)
        _check(lib().kde_batch_run_async(self.handle, wp, wn, _stream_handle(stream)))

    def results(self):
        out = (kde_result * self.n)()
        _check(lib().kde_batch_results(self.handle, out))
        return [r.as_dict() for r in out]

    def g(self, ws, req: int, n_h: int) -> np.ndarray:
        out = np.zeros(n_h)
        _check(lib().kde_batch_g(self.handle, ctypes.c_void_p(ws.data_ptr()), int(req), _dp(out)))
        return out

    def close(self):
        if self.handle:
            lib().kde_batch_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kde_batch_workspace_size(requests, opts: kde_opts | None = None) -> int:
    arr = (kde_request * len(requests))(*requests)
    out = ctypes.c_size_t(0)
    _check(lib().kde_batch_workspace_size(arr, len(requests), ctypes.byref(opts) if opts else None,
                                          ctypes.byref(out)))
    return out.value


def kde_select_batch(requests, opts: kde_opts | None = None, ws=None, stream=None):
    arr = (kde_request * len(requests))(*requests)
    if ws is None:
        ws = workspace(kde_batch_workspace_size(requests, opts))
    wp, wn = _ws(ws)
    out = (kde_result * len(requests))()
    _check(lib().kde_select_batch(arr, len(requests), ctypes.byref(opts) if opts else None, wp, wn,
                                  _stream_handle(stream), out))
    return [r.as_dict() for r in out]


# ------------------------------------------------------------------ serving

class Server:
    """kde_serve_*: a continuous-batching server over a caller-owned arena
    (a torch uint8 tensor whose size is the HBM budget)."""

    def __init__(self, arena, max_slots=256, max_queue=0, quantum_evals=0.0, step_deadline_ms=0,
                 device=0, opts: kde_opts | None = None):
        self.arena = arena
        self._opts = opts
        cfg = kde_serve_config(ctypes.c_void_p(arena.data_ptr()), arena.numel(), int(max_slots),
                               int(max_queue), float(quantum_evals), int(step_deadline_ms),
                               int(device), ctypes.pointer(opts) if opts else None)
        h = ctypes.c_void_p(0)
        _check(lib().kde_serve_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h

    def submit(self, x_host: np.ndarray, methods: int, grid: kde_grid | None = None) -> int:
        req, _keep = make_request(np.ascontiguousarray(x_host), methods, grid)
        t = ctypes.c_uint64(0)
        _check(lib().kde_serve_submit(self.handle, ctypes.byref(req), ctypes.byref(t)))
        return t.value

    def submit_status(self, x_host: np.ndarray, methods: int, grid: kde_grid | None = None):
        """(status, ticket) without raising."""
        req, _keep = make_request(np.ascontiguousarray(x_host), methods, grid)
        t = ctypes.c_uint64(0)
        rc = lib().kde_serve_submit(self.handle, ctypes.byref(req), ctypes.byref(t))
        return rc, t.value

    def poll(self, ticket: int):
        """(status, result dict); status KDE_EAGAIN while not finished."""
        res = kde_result()
        rc = lib().kde_serve_poll(self.handle, ctypes.c_uint64(ticket), ctypes.byref(res))
        return rc, res.as_dict()

    def wait(self, ticket: int, timeout_ms: int = -1):
        res = kde_result()
        rc = lib().kde_serve_wait(self.handle, ctypes.c_uint64(ticket), int(timeout_ms),
                                  ctypes.byref(res))
        return rc, res.as_dict()

    def cancel(self, ticket: int) -> int:
        return lib().kde_serve_cancel(self.handle, ctypes.c_uint64(ticket))

    def stats(self) -> dict:
        s = kde_serve_stats_t()
        _check(lib().kde_serve_stats(self.handle, ctypes.byref(s)))
        return s.as_dict()

    def close(self):
        if self.handle:
            lib().kde_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
