"""The continuous-batching server (kde_serve_*) through the C ABI.

Failure detection is exercised on the host only: a step deadline that the
host declares missed, cancellation, a full queue, an oversized request.  No
test faults, traps or stalls the GPU."""
import time

import numpy as np
import pytest

import oracle
from paper_1505_01998_gb300 import datagen
from tests._helpers import TOL, argmin_ok, built_lib, g_err, lscv_A

pytestmark = pytest.mark.gpu

LSCV, PLUGIN = 1, 2


@pytest.fixture(scope="module")
def kde():
    return built_lib()


def arena(nbytes):
    from paper_1505_01998_gb300 import gbkde
    return gbkde.workspace(nbytes)


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _requests(count, seed, lo=800, hi=20000):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        d = 1 if rng.uniform() < 0.8 else 2
        methods = LSCV if d == 2 else (PLUGIN if rng.uniform() < 0.6 else LSCV)
        x = datagen.correlated_mixture(n, d, seed=int(rng.integers(1 << 30)))
        out.append((x, methods))
    return out


def _single(kde, x, methods, grid):
    if methods == LSCV:
        return kde.kde_lscv(dev(x), grid)[0]
    return kde.kde_plugin(dev(x))


def _oracle_check(r, x, methods, n_h):
    """A served result against the FP64 oracle on the request's own samples:
    LSCV g at the served index within 1e-5 of the oracle's g (scaled as in the
    parity tests), the index the oracle's first minimum or a certified near
    tie, h the grid point; PLUGIN psi6/psi4 within 1e-5 of their magnitude
    scale, g2 and h within 1e-5 relative (Sec. 4.4.1 and 4.4.2)."""
    x64 = np.asarray(x, dtype=np.float64)
    if x64.ndim == 1:
        x64 = x64[None, :]
    d, n = x64.shape
    if methods & LSCV:
        h = oracle.grid_default(n, d, n_h)
        ref = oracle.lscv_h(x64, h)
        k = r["argmin"]
        A = lscv_A(x64)
        err = g_err(r["g_min"], ref["g"][k], ref["s_kk"][k], ref["s_k"][k], h[k], n, d, A)
        assert err <= TOL, (n, d, k, r["g_min"], ref["g"][k])
        tol_abs = TOL * float(np.max(np.abs(ref["g"])))
        assert argmin_ok(k, ref["g"], tol_abs), (k, int(np.argmin(ref["g"])))
        assert abs(r["h"] - h[k]) <= 1e-12 * h[k]
    if methods & PLUGIN:
        ref = oracle.plugin(x64[0])
        assert ref["status"] == 0
        for key, rr, gk in (("psi6", 6, "g1"), ("psi4", 4, "g2")):
            g = ref[gk]
            mag = (2 * oracle.psi_abs_pair_sum(x64[0], rr, g) + n * abs(oracle.gauss_deriv(rr, 0.0))) / (
                n * n * g ** (rr + 1))
            assert abs(r[key] - ref[key]) <= TOL * max(abs(ref[key]), mag), (key, r[key], ref[key])
        assert abs(r["g2"] - ref["g2"]) <= TOL * ref["g2"]
        hp = r["h_plugin"] if methods & LSCV else r["h"]
        assert abs(hp - ref["h"]) <= TOL * ref["h"], (hp, ref["h"])


def test_results_in_the_mix_equal_alone_bitwise_and_single_calls_within_tolerance(kde):
    """40 requests on the device together: each result equals the same request
    served alone (bitwise), the single call (within 1e-5) and the FP64 oracle
    on that request's samples (within 1e-5)."""
    grid = kde.make_grid(n_h=128)[0]
    reqs = _requests(40, seed=1, lo=600, hi=6000)
    srv = kde.Server(arena(1 << 30), max_slots=64)
    tickets = [srv.submit(x, m, grid) for x, m in reqs]
    outs = []
    for t in tickets:
        rc, r = srv.wait(t, 60000)
        assert rc == 0, (rc, r)
        outs.append(r)
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["active_max"] > 1  # requests were on the device together
    alone = kde.Server(arena(1 << 30), max_slots=1)  # the same requests one at a time
    for (x, m), r in zip(reqs, outs):
        rc, a = alone.wait(alone.submit(x, m, grid), 60000)
        assert rc == 0
        assert a == r  # bitwise, every field
        s = _single(kde, x, m, grid)
        if m == LSCV:
            assert r["argmin"] == s["argmin"] and r["h"] == s["h"]
            assert abs(r["g_min"] - s["g_min"]) <= 1e-5 * abs(s["g_min"])
        else:
            for k in ("psi6", "g2", "psi4", "h"):
                assert abs(r[k] - s[k]) <= 1e-5 * abs(s[k]), (k, r[k], s[k])
        _oracle_check(r, x, m, 128)
    alone.close()


def test_wide_samples_on_one_and_two_point_grids_in_the_mix(kde):
    """Requests of d = 6 and 16 on one- and two-point grids (warp items) served
    beside d = 1 requests on the default grid, with steps small enough that
    every request spans several: each result equals the single call's."""
    rng = np.random.default_rng(31)
    mix = []
    for k in range(12):
        d = [16, 6, 1][k % 3]
        n = int(rng.integers(900, 5000))
        x = datagen.correlated_mixture(n, d, seed=900 + k)
        if d == 1:
            grid, hk = kde.make_grid(n_h=128)
        else:
            h = oracle.grid_default(n, d, 8)[3:3 + 1 + k % 2]
            grid, hk = kde.make_grid(h=h)
        mix.append((x, grid, hk))
    srv = kde.Server(arena(1 << 30), max_slots=16, quantum_evals=2e8)
    tickets = [srv.submit(x, LSCV, grid) for x, grid, _ in mix]
    for t, (x, grid, _) in zip(tickets, mix):
        rc, r = srv.wait(t, 60000)
        assert rc == 0, (rc, r)
        s = kde.kde_lscv(dev(x), grid)[0]
        assert r["argmin"] == s["argmin"] and r["h"] == s["h"]
        assert abs(r["g_min"] - s["g_min"]) <= 1e-5 * abs(s["g_min"])
    srv.close()


@pytest.mark.parametrize("quantum", [3e8, 2e9])
def test_phases_spanning_many_steps_match_single_calls(kde, quantum):
    """Small step budgets split every phase of every request over many steps,
    two of them in flight: each result (including LSCV + PLUGIN requests,
    whose PLUGIN phases follow the LSCV phase) must equal the single calls
    within tolerance -- a phase's result is taken only from the step that ran
    its finishing kernels."""
    grid = kde.make_grid(n_h=64)[0]
    rng = np.random.default_rng(7)
    reqs = []
    for k in range(14):
        n = int(rng.integers(3000, 24000))
        d = 2 if k % 5 == 4 else 1
        methods = LSCV if d == 2 else [LSCV, PLUGIN, LSCV | PLUGIN][k % 3]
        reqs.append((datagen.correlated_mixture(n, d, seed=900 + k), methods))
    srv = kde.Server(arena(1 << 30), max_slots=16, quantum_evals=quantum)
    tickets = [srv.submit(x, m, grid) for x, m in reqs]
    outs = []
    for t in tickets:
        rc, r = srv.wait(t, 120000)
        assert rc == 0, (rc, r)
        outs.append(r)
    st = srv.stats()
    srv.close()
    assert st["steps"] > 2 * len(reqs)
    for (x, m), r in zip(reqs, outs):
        if m & LSCV:
            s = kde.kde_lscv(dev(x), grid)[0]
            assert r["argmin"] == s["argmin"], (r, s)
            assert abs(r["g_min"] - s["g_min"]) <= 1e-5 * abs(s["g_min"])
        if m & PLUGIN:
            s = kde.kde_plugin(dev(x))
            for k in ("psi6", "g2", "psi4", "h_plugin"):
                assert abs(r[k] - s[k]) <= 1e-5 * abs(s[k]), (k, r[k], s[k])
            if not (m & LSCV):
                assert abs(r["h"] - s["h"]) <= 1e-5 * abs(s["h"])
        if x.shape[-1] <= 8000:
            _oracle_check(r, x, m, 64)


def test_admission_under_a_small_budget(kde):
    grid = kde.make_grid(n_h=64)[0]
    reqs = _requests(30, seed=2, lo=2000, hi=30000)
    budget = 24 << 20
    srv = kde.Server(arena(budget), max_slots=32)
    tickets = [srv.submit(x, m, grid) for x, m in reqs]
    for t in tickets:
        rc, r = srv.wait(t, 120000)
        assert rc == 0
    st = srv.stats()
    srv.close()
    assert st["completed"] == 30
    assert st["arena_peak_bytes"] <= budget
    assert st["queue_depth_max"] > 0 and st["p99_wait_ms"] > 0  # some had to wait for memory


def test_cancel_queued_and_running(kde):
    grid = kde.make_grid(n_h=256)[0]
    big = datagen.skewed_column(65536, seed=9)
    small = datagen.mixture_1d(3000, seed=3).astype(np.float32)
    # one slot: the second request queues.  A cancel takes effect at the next
    # step boundary (the two steps in flight run to their end), so the step
    # budget keeps the big request (5.5e11 evaluations) spread over ~6 steps.
    srv = kde.Server(arena(1 << 30), max_slots=1, quantum_evals=5e10)
    t_big = srv.submit(big, LSCV, grid)
    t_q = srv.submit(small, LSCV, grid)
    t_ok = srv.submit(small, PLUGIN)
    assert srv.cancel(t_q) == 0
    assert srv.cancel(t_big) == 0
    rc, r = srv.wait(t_q, 10000)
    assert rc == kde.KDE_ECANCELLED
    rc, r = srv.wait(t_big, 60000)
    assert rc == kde.KDE_ECANCELLED
    rc, r = srv.wait(t_ok, 60000)
    assert rc == 0
    assert abs(r["h"] - kde.kde_plugin(dev(small))["h"]) <= 1e-5 * r["h"]
    st = srv.stats()
    srv.close()
    assert st["cancelled"] == 2 and st["completed"] == 1


def test_step_deadline_fails_requests_on_the_host_and_server_recovers(kde):
    grid = kde.make_grid(n_h=256)[0]
    big = datagen.skewed_column(65536, seed=4)
    # one step of this request is ~tens of ms; a 1 ms deadline is missed
    srv = kde.Server(arena(1 << 30), max_slots=4, quantum_evals=5e11, step_deadline_ms=1)
    t = srv.submit(big, LSCV, grid)
    rc, r = srv.wait(t, 60000)
    assert rc == kde.KDE_ETIMEDOUT
    srv.close()
    # a fresh server on the same device keeps serving correctly
    srv = kde.Server(arena(256 << 20), max_slots=4)
    x = datagen.mixture_1d(5000, seed=5).astype(np.float32)
    rc, r = srv.wait(srv.submit(x, PLUGIN), 60000)
    srv.close()
    assert rc == 0 and abs(r["h"] - kde.kde_plugin(dev(x))["h"]) <= 1e-5 * r["h"]


def test_busy_and_wait_timeout(kde):
    grid = kde.make_grid(n_h=128)[0]
    srv = kde.Server(arena(4 << 20), max_slots=2, max_queue=1)
    huge = datagen.correlated_mixture(262144, 4, seed=1)  # 8 MB of staged samples alone
    rc, _ = srv.submit_status(huge, LSCV, grid)
    assert rc == kde.KDE_EBUSY  # alone larger than the arena
    x = datagen.mixture_1d(20000, seed=2).astype(np.float32)
    t1 = srv.submit(x, LSCV, grid)
    rc, _ = srv.wait(t1, 0)
    assert rc in (0, kde.KDE_ETIMEDOUT)
    for t in [t1]:
        rc, r = srv.wait(t, 60000)
        assert rc == 0
    rc, r = srv.poll(123456)
    assert rc == kde.KDE_ENOTFOUND
    srv.close()
