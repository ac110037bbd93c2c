#!/usr/bin/env python
"""Benchmark of exact KDE bandwidth selection on GB300 (arXiv 1505.01998).

Metric: pair-bandwidth kernel evaluations per second.  One evaluation is one
(pair i<j, bandwidth) term: an LSCV_h term for every grid point, or a psi_r
term of the PLUGIN method.  One step = one LSCV_h selection on a 256-point
grid over Z(h0) plus one PLUGIN selection (psi_6 and psi_4 over all pairs) of
the n = 65,536 skewed column (half lognormal(0,1), half U[0,100], seed 2 +
rank): P = n(n-1)/2 pairs, 258 P evaluations per step.

  value     device time of K steps, samples resident in HBM (CUDA events)
  e2e       the same selections through the host-buffer entry points:
            pinned host samples in, results out, host wall clock
  roofline  the all-pairs LSCV kernel timed live with CUDA events around its
            launch, against its ALU roofline (MUFU ex2 and FP32 lanes per
            evaluation, unit rates measured by kde_probe_alu) x SMs x the SM
            clock sampled during the timed region
  cpu_baseline  the FP64 oracle on a bounded sample (rows of the pair
            triangle, the same 256-point grid) on the host's cores

--impl reference times the oracle alone (the reference arm).
Multi-GPU (torchrun): every rank selects its own replica dataset (weak
scaling, no collective on the data path); value = all ranks' evaluations
divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 65536
N_H = 256
SEED = 2
METRIC = "pair-bandwidth kernel evals/s"
UNIT = "evals/s"
WORKLOAD = ("skewed column n=65536 FP32 (lognormal(0,1) + U[0,100]); LSCV_h on a 256-point "
            "log grid over Z(h0) + two-stage PLUGIN (psi_6, psi_4)")


def pairs(n):
    return n * (n - 1) // 2


EVALS_LSCV = pairs(N) * N_H
EVALS_PSI = 2 * pairs(N)
EVALS_STEP = EVALS_LSCV + EVALS_PSI


def lscv_per_clk(probe, d, octave):
    """ALU bound of the LSCV pair kernel in evaluations per clock and SM.
    Direct grids: one ex2 and 3 FP32 lane-operations per evaluation (the
    squared distance, 2d lanes per pair, is shared by 16 bandwidths and left
    out).  Octave grids, per 16 evaluations (one pair, two residues, eight
    octaves): 6 ex2; one scaling, 3 squarings and 6 running sums in
    FMUL2/FADD2 (20 lanes; the other two scalings are exponent adds on the
    integer pipe); 3 squarings fused with their running sums in FFMA2
    (6 lanes); and 2d FMA lanes for the squared distance."""
    if not octave:
        return min(probe["mufu_ex2_per_clk_sm"], probe["ffma_lanes_per_clk_sm"] / 3.0)
    fp32 = 1.0 / (1.25 / probe["fmul2_fadd2_lanes_per_clk_sm"] + 0.375 / probe["ffma2_lanes_per_clk_sm"]
                  + (2.0 * d / 16.0) / probe["ffma_lanes_per_clk_sm"])
    return min(probe["mufu_ex2_per_clk_sm"] / 0.375, fp32)


def lscv_basis(probe, d, octave, mhz):
    if not octave:
        return (f"min(MUFU ex2 {probe['mufu_ex2_per_clk_sm']:.1f}/clk/SM, FP32 lanes "
                f"{probe['ffma_lanes_per_clk_sm']:.1f}/clk/SM / 3 per eval) x {probe['sm_count']} SMs x "
                f"{mhz:.0f} MHz")
    return (f"octave grid: min(MUFU ex2 {probe['mufu_ex2_per_clk_sm']:.1f}/clk/SM / 0.375 per eval, "
            f"1 / (1.25 / {probe['fmul2_fadd2_lanes_per_clk_sm']:.1f} FMUL2/FADD2 lanes + 0.375 / "
            f"{probe['ffma2_lanes_per_clk_sm']:.1f} FFMA2 lanes + {2 * d}/16 / "
            f"{probe['ffma_lanes_per_clk_sm']:.1f} FFMA lanes) per eval) x "
            f"{probe['sm_count']} SMs x {mhz:.0f} MHz")


def set_n(n):
    global N, EVALS_LSCV, EVALS_PSI, EVALS_STEP, WORKLOAD
    if n != N:
        WORKLOAD = WORKLOAD.replace(f"n={N}", f"n={n}")
    N = n
    EVALS_LSCV = pairs(N) * N_H
    EVALS_PSI = 2 * pairs(N)
    EVALS_STEP = EVALS_LSCV + EVALS_PSI
# LSCV: setup, prologue statistics, whitening, pairs, reduce, finish (the
# n = 65,536 partial table is too large for the pair kernel to finish itself);
# PLUGIN: setup, prologue statistics, whitening, 2 x pairs (each finished by
# its last CTA)
LAUNCHES_PER_STEP = 6 + 5


def profiled_lscv_traffic():
    """DRAM bytes per full-size launch of the LSCV kernel from the committed ncu
    summary, or None when the kernel source changed since that capture."""
    import hashlib
    import re
    prof = os.path.join(ROOT, "profiles", "k_lscv_skewed_column.md")
    src = os.path.join(ROOT, "paper_1505_01998_gb300", "csrc", "lscv.cu")
    try:
        text = open(prof).read()
        want = re.search(r"sha256 prefix\s+`([0-9a-f]{16})`", text).group(1)
        have = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        if want != have or N != 65536:
            return None
        return int(re.search(r"traffic\s+=\s+([0-9,]+)\s+bytes", text).group(1).replace(",", ""))
    except Exception:
        return None


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        with open(self.path) as fh:
            lines = fh.readlines()
        os.unlink(self.path)
        return parse_clock_samples(lines)


def parse_clock_samples(lines):
    """Summary of `nvidia-smi --query-gpu=<ClockSampler.FIELDS> --format=csv,noheader,nounits`
    lines: median SM clock over the loaded samples (at least half the highest
    clock seen), the maximum clock, the throttle reasons seen active, the
    sample count and the highest power draw; None without samples."""
    rows = []
    for line in lines:
        p = [s.strip() for s in line.split(",")]
        if len(p) >= 9 and p[1].replace(".", "").isdigit():
            rows.append(p)
    if not rows:
        return None
    sm = [float(r[1]) for r in rows]
    names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
    reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
    loaded = [s for s in sm if s >= 0.5 * max(sm)] or sm
    return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": float(rows[0][2]),
            "reasons": reasons, "samples": len(rows),
            "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
            if any(r[3].replace(".", "").isdigit() for r in rows) else None}


# --------------------------------------------------------------- oracle leg

def oracle_sample(seconds: float, rank_seed: int = SEED):
    """Time the FP64 oracle on a bounded sample of the same workload: LSCV
    pair sums for rows [0, m) of the pair triangle against all later samples,
    on the 256-point grid.  m is calibrated to take about `seconds`."""
    import numpy as np

    import oracle
    from paper_1505_01998_gb300 import datagen

    x = datagen.skewed_column(N, seed=rank_seed).astype(np.float64)
    h = oracle.grid_default(N, 1, N_H)
    cores = oracle.openmp_threads() or 1
    t0 = time.perf_counter()
    oracle.lscv_sums(x, h, block=(0, 2 * cores, 0, N))
    dt = time.perf_counter() - t0
    rate_rows = 2 * cores / max(dt, 1e-6)
    m = int(max(cores, min(N - 1, rate_rows * seconds)))
    t0 = time.perf_counter()
    oracle.lscv_sums(x, h, block=(0, m, 0, N))
    dt = time.perf_counter() - t0
    npairs = sum(N - 1 - i for i in range(m))
    return {"value": npairs * N_H / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"LSCV_h pair sums of rows 0..{m - 1} of the n={N} pair triangle "
                      f"({npairs} pairs x {N_H} bandwidths, FP64, {dt:.1f} s)",
            "seconds": dt}


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    budget = 150.0 / max(1, args.steps + args.warmup)
    for _ in range(args.warmup):
        oracle_sample(min(budget, 3.0))
    vals, secs = [], []
    for _ in range(args.steps):
        r = oracle_sample(budget)
        vals.append(r["value"])
        secs.append(r["seconds"])
    v = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(secs), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N, "d": 1, "n_h": N_H, "seed": SEED,
                       "sample": "rows of the pair triangle per step (bounded oracle sample)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                             "sample": r["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------- batch and serving

def run_batch(args):
    """512 univariate datasets (sizes log-uniform on [256, 131072], seed 4),
    each LSCV on 128 points over Z(h0) plus PLUGIN, as one graph-captured batch;
    against the plain per-dataset path (one kde_lscv + kde_plugin pair of
    calls per dataset on one stream)."""
    import torch
    torch.cuda.set_device(0)
    print(json.dumps(batch_measure(args.batch_count, args.steps, args.warmup, args.autotune)), flush=True)
    return 0


def batch_measure(count, steps, warmup, autotune=False):
    import numpy as np
    import torch

    from paper_1505_01998_gb300 import datagen, gbkde

    sets = datagen.batch(count, seed=4)
    xs = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in sets]
    grid = gbkde.make_grid(n_h=128)[0]
    reqs, keep = [], []
    for x in xs:
        r, k = gbkde.make_request(x, gbkde.KDE_METHOD_LSCV | gbkde.KDE_METHOD_PLUGIN, grid)
        reqs.append(r)
        keep.append(k)
    evals = sum(pairs(x.shape[1]) * (128 + 2) for x in xs)
    tuned = {}
    if autotune:
        # tune the size buckets where geometry matters (n <= 16384); larger
        # datasets fill the GPU on their own and keep the default rules
        by_bucket = {}
        for x in xs:
            n = x.shape[1]
            b = int(math.ceil(math.log2(n)))
            if n <= 16384 and (b not in by_bucket or n > by_bucket[b].shape[1]):
                by_bucket[b] = x
        tws = gbkde.workspace(2 << 30)
        for b, x in sorted(by_bucket.items()):
            o, rate = gbkde.kde_autotune(x, 128, gbkde.KDE_TUNE_THROUGHPUT, tws)
            tuned[b] = {"tile": o.tile, "bw_per_thread": o.bw_per_thread, "ctas_per_sm": o.ctas_per_sm,
                        "tiles_per_item": o.tiles_per_item, "evals_per_s": rate}
        del tws
    plan = gbkde.BatchPlan(reqs, keepalive=keep)
    ws = gbkde.workspace(plan.ws_bytes)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(max(1, warmup)):
        plan.run(ws)
    ms = []
    for _ in range(steps):
        e0.record(stream)
        plan.run_async(ws, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    res = plan.results()
    # plain per-dataset path
    wss = [gbkde.workspace(max(gbkde.kde_workspace_size(x.shape[1], 1, 128),
                               gbkde.kde_workspace_size(x.shape[1], 1, 0))) for x in xs]
    wsp = [gbkde.workspace(gbkde.kde_workspace_size(x.shape[1], 1, 0)) for x in xs]

    def plain():
        for x, w, wp in zip(xs, wss, wsp):
            gbkde.kde_lscv_async(x, grid, None, w, stream)
            gbkde.kde_plugin_async(x, None, wp, stream)

    plain()
    torch.cuda.synchronize()
    pms = []
    for _ in range(max(1, steps // 2)):
        e0.record(stream)
        plain()
        e1.record(stream)
        torch.cuda.synchronize()
        pms.append(e0.elapsed_time(e1))
    # equal results: the plain path's last result of every dataset
    same = all(gbkde.read_ws_result(w, 128)[0]["g_min"] == r["g_min"] for w, r in zip(wss, res))
    t = statistics.median(ms)
    line = {"workload": "batch", "metric": METRIC + " (batched, CUDA-graph replay)", "unit": UNIT,
            "value": evals / (t * 1e-3), "ms_per_batch": t, "datasets": len(xs),
            "evals_per_batch": evals, "samples": int(sum(x.shape[1] for x in xs)),
            "plain_path": {"value": evals / (statistics.median(pms) * 1e-3),
                           "ms_per_batch": statistics.median(pms)},
            "speedup_vs_plain": statistics.median(pms) / t,
            "bitwise_equal_to_plain": bool(same),
            "statuses_ok": sum(r["status"] == 0 for r in res),
            "autotuned_buckets": tuned}
    plan.close()
    return line


def run_serve(args):
    """Poisson arrivals of selection requests (n log-uniform on [1024, 262144],
    d = 1 : 2 at 4 : 1, LSCV or PLUGIN half and half) at a sweep of rates,
    served under a 40 GB arena; against the plain path (the same requests,
    one kde_lscv / kde_plugin call at a time in arrival order)."""
    import torch
    torch.cuda.set_device(0)
    out = serve_measure(args.rates, args.serve_count, args.serve_seeds, args.serve_budget_gb,
                        args.serve_quantum, verbose=True)
    print(json.dumps(dict({"workload": "serve", "metric": "served selections/s", "unit": "requests/s"}, **out)),
          flush=True)
    return 0


def serve_measure(rates, count, seeds, budget_gb, quantum, verbose=False, repeat_from_rate=0.0):
    """Serve `count` requests at each rate for each arrival seed, then the same
    requests through the plain path.  Per rate: served and plain requests/s,
    p50 and p99 latency (median and range over the seeds), and agreement of
    every request's selected bandwidth between the two paths.  Rates below
    `repeat_from_rate` run the first seed only."""
    import numpy as np
    import torch

    from paper_1505_01998_gb300 import datagen, gbkde

    grid = gbkde.make_grid(n_h=128)[0]
    arena = gbkde.workspace(budget_gb << 30)
    stream = torch.cuda.current_stream()
    records = []
    for rate in rates:
        runs = []
        for seed in (seeds if rate >= repeat_from_rate else seeds[:1]):
            reqs = datagen.serving_requests(rate, count, seed=seed)
            runs.append(_serve_once(gbkde, torch, np, reqs, grid, arena, stream, quantum))
            if verbose:
                print(json.dumps(dict({"rate": rate, "seed": seed}, **runs[-1])), flush=True)
        rec = {"rate": rate, "requests": count, "seeds": list(seeds if rate >= repeat_from_rate else seeds[:1])}
        for side in ("served", "plain"):
            rec[side] = {}
            for key in ("requests_per_s", "p50_ms", "p99_ms"):
                v = [r[side][key] for r in runs]
                rec[side][key] = statistics.median(v)
                if len(v) > 1:
                    rec[side][key + "_range"] = [min(v), max(v)]
        rec["served"]["active_max"] = max(r["served"]["active_max"] for r in runs)
        rec["agreement"] = {"requests": sum(r["agreement"]["requests"] for r in runs),
                            "max_rel_diff_h": max(r["agreement"]["max_rel_diff_h"] for r in runs),
                            "lscv_argmin_differs": sum(r["agreement"]["lscv_argmin_differs"] for r in runs),
                            "lscv_argmin_near_ties": sum(r["agreement"]["lscv_argmin_near_ties"] for r in runs),
                            "lscv_argmin_gap_rel_max": max(r["agreement"]["lscv_argmin_gap_rel_max"]
                                                           for r in runs),
                            "failures": sum(len(r["failures"]) for r in runs)}
        records.append(rec)
    best = max(r["served"]["requests_per_s"] for r in records)
    best_plain = max(r["plain"]["requests_per_s"] for r in records)
    return {"value": best, "plain_path_value": best_plain, "budget_bytes": budget_gb << 30,
            "quantum_evals": quantum, "rates": records}


def _serve_once(gbkde, torch, np, reqs, grid, arena, stream, quantum):
    srv = gbkde.Server(arena, max_slots=256, quantum_evals=quantum)
    t0 = time.perf_counter()
    tickets = []
    for r in reqs:
        now = time.perf_counter() - t0
        if r.arrival_s > now:
            time.sleep(r.arrival_s - now)
        m = gbkde.KDE_METHOD_LSCV if r.method == "lscv" else gbkde.KDE_METHOD_PLUGIN
        tickets.append(srv.submit(r.x, m, grid))
    failures = []
    served_res = {}
    keys = ("sigma", "g1", "psi6", "g2", "psi4", "h", "argmin", "g_min", "logdet_S")
    for k, t in enumerate(tickets):
        rc, res = srv.wait(t, 600000)
        if rc != 0:
            r = reqs[k]
            failures.append({"index": k, "status": rc, "n": r.n, "d": r.d, "method": r.method,
                             "seed": r.seed, "served": {q: res.get(q) for q in keys}})
        else:
            served_res[k] = res
    st = srv.stats()
    srv.close()
    # plain path: arrivals at the same times, served one at a time
    ws = gbkde.workspace(max(gbkde.kde_workspace_size(r.n, r.d, 128) for r in reqs))
    lat = []
    plain_fail = {}
    plain_res = {}
    plain_g = {}
    t0 = time.perf_counter()
    for k, r in enumerate(reqs):
        now = time.perf_counter() - t0
        if r.arrival_s > now:
            time.sleep(r.arrival_s - now)
        xd = torch.from_numpy(r.x).cuda()
        try:
            if r.method == "lscv":
                plain_res[k], plain_g[k], _ = gbkde.kde_lscv(xd, grid, None, ws, stream)
            else:
                plain_res[k] = gbkde.kde_plugin(xd, None, ws, stream)
        except gbkde.KdeError as e:
            plain_fail[k] = e.status
        lat.append(1e3 * (time.perf_counter() - t0 - r.arrival_s))
    span = time.perf_counter() - t0
    del ws
    for f in failures:  # the same request through the single-call path
        f["plain_status"] = plain_fail.get(f["index"], 0)
        if f["index"] in plain_res:
            f["plain"] = {q: plain_res[f["index"]].get(q) for q in keys}
    # equal accuracy: the selected bandwidth of every request served on both paths
    both = [k for k in served_res if k in plain_res]
    h_rel = max((abs(served_res[k]["h"] - plain_res[k]["h"]) / abs(plain_res[k]["h"]) for k in both),
                default=0.0)
    differ = [k for k in both if reqs[k].method == "lscv"
              and served_res[k]["argmin"] != plain_res[k]["argmin"]]
    # a differing grid index is a near tie when the single call's own g at the
    # served index is within the g tolerance (1e-5 of |g|) of its minimum: the
    # two summation groupings (served items are capped in size) round apart
    gaps = [(plain_g[k][served_res[k]["argmin"]] - plain_g[k][plain_res[k]["argmin"]])
            / abs(plain_g[k][plain_res[k]["argmin"]]) for k in differ]
    return {"failures": failures,
            "agreement": {"requests": len(both), "max_rel_diff_h": h_rel,
                          "lscv_argmin_differs": len(differ),
                          "lscv_argmin_near_ties": int(sum(bool(g <= 1e-5) for g in gaps)),
                          "lscv_argmin_gap_rel_max": float(max(gaps, default=0.0)),
                          "lscv_argmin_differing": [
                              {"n": int(reqs[k].n), "d": int(reqs[k].d),
                               "served": int(served_res[k]["argmin"]),
                               "single_call": int(plain_res[k]["argmin"]), "gap_rel": float(g)}
                              for k, g in zip(differ, gaps)]},
            "served": {"requests_per_s": st["requests_per_s"], "p50_ms": st["p50_ms"],
                       "p99_ms": st["p99_ms"], "p50_wait_ms": st["p50_wait_ms"],
                       "evals_per_s": st["evals_per_s"], "active_max": st["active_max"],
                       "steps": st["steps"], "arena_peak_bytes": st["arena_peak_bytes"]},
            "plain": {"requests_per_s": len(reqs) / span,
                      "p50_ms": float(np.percentile(lat, 50)),
                      "p99_ms": float(np.percentile(lat, 99))}}


def run_paper(args):
    """The largest instances of the paper's experiments (Sec. 7.2, Table 1),
    timed end to end (host samples in, results out, as the paper timed its
    GPU runs) and with samples resident; the paper's GTX 480 times are quoted
    as context."""
    import numpy as np
    import torch

    from paper_1505_01998_gb300 import datagen, gbkde

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    out = []

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        return 1e3 * statistics.median(ts)

    def plan_timed(xd, methods, grid, reps):
        """The same selection as a batch plan built once and replayed (one
        captured graph per run), samples resident."""
        req, keep = gbkde.make_request(xd, methods, grid)
        plan = gbkde.BatchPlan([req], keepalive=[keep])
        wsp = gbkde.workspace(plan.ws_bytes)
        ms = timed(lambda: plan.run(wsp, stream), reps)
        assert plan.run(wsp, stream)[0]["status"] == 0
        return ms

    # PLUGIN, n = 32768, d = 1 (paper: 87.9 ms)
    x = datagen.mixture_1d(32768, seed=7).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    ws = gbkde.workspace(gbkde.kde_workspace_size(32768, 1, 0))
    xh = torch.from_numpy(x).pin_memory().numpy()
    e2e = timed(lambda: gbkde.kde_plugin_host(xh, None, ws, stream), args.steps)
    res = timed(lambda: gbkde.kde_plugin(xd, None, ws, stream), args.steps)
    plan_ms = plan_timed(xd, gbkde.KDE_METHOD_PLUGIN, None, args.steps)
    out.append({"instance": "PLUGIN n=32768 d=1", "e2e_ms": e2e, "resident_ms": res,
                "resident_plan_ms": plan_ms,
                "paper_gpu_ms": 87.9, "paper_sse_ms": 1442.3, "paper_seq_ms": 47435.3,
                "speedup_vs_paper_gpu_e2e": 87.9 / e2e})
    # LSCV_h, n = 1024, d = 16, 150 bandwidths (paper: 14.7 ms)
    x = datagen.correlated_mixture(1024, 16, seed=8)
    xd = torch.from_numpy(x).cuda()
    grid = gbkde.make_grid(n_h=150)[0]
    ws = gbkde.workspace(gbkde.kde_workspace_size(1024, 16, 150))
    xh = torch.from_numpy(x).pin_memory().numpy()
    e2e = timed(lambda: gbkde.kde_lscv_host(xh, grid, None, ws, stream), args.steps)
    res = timed(lambda: gbkde.kde_lscv(xd, grid, None, ws, stream), args.steps)
    plan_ms = plan_timed(xd, gbkde.KDE_METHOD_LSCV, grid, args.steps)
    out.append({"instance": "LSCV_h n=1024 d=16 n_h=150", "e2e_ms": e2e, "resident_ms": res,
                "resident_plan_ms": plan_ms,
                "paper_gpu_ms": 14.7, "paper_sse_ms": 344.1, "paper_seq_ms": 8283.6,
                "speedup_vs_paper_gpu_e2e": 14.7 / e2e})
    # LSCV_H, one g(H), n = 16384, d = 16 (paper: 184.2 ms)
    x = datagen.correlated_mixture(16384, 16, seed=9)
    xd = torch.from_numpy(x).cuda()
    S = gbkde.kde_sample_covariance(xd)
    H = (0.5 * S)[None]
    ws = gbkde.workspace(gbkde.kde_lscv_H_workspace_size(16384, 16, 1))
    xh = torch.from_numpy(x).pin_memory()

    def lscv_H_e2e():
        xd2 = xh.cuda(non_blocking=True)
        gbkde.kde_lscv_H(xd2, H, None, ws, stream)

    e2e = timed(lscv_H_e2e, args.steps)
    res = timed(lambda: gbkde.kde_lscv_H(xd, H, None, ws, stream), args.steps)
    out.append({"instance": "LSCV_H g(H) n=16384 d=16", "e2e_ms": e2e, "resident_ms": res,
                "paper_gpu_ms": 184.2, "paper_sse_ms": 2320.0, "paper_seq_ms": 53258.8,
                "speedup_vs_paper_gpu_e2e": 184.2 / e2e})
    print(json.dumps({"workload": "paper_table1", "note": "paper times: GTX 480 / Core i7 SSE / "
                      "sequential C, FP32, transfers included (Sec. 7.1-7.3, Table 1)",
                      "instances": out}), flush=True)
    return 0


def run_configs(args):
    """The n = 1,024 FP64 mixture (64-point grid on [0.01, 2] + plug-in) and
    the d = 2, 3, 4, n = 16,384 correlated mixtures (128-point grid over
    Z(h0)): GPU rate with samples resident (CUDA events around the LSCV
    kernel, and around the whole selection), end to end from host samples,
    and the FP64 oracle on the host cores (in full for n = 1,024, on rows of
    the pair triangle for the d > 1 sets)."""
    import numpy as np
    import torch

    import oracle
    from paper_1505_01998_gb300 import datagen, gbkde

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    probe = gbkde.kde_probe_alu()
    peak = lscv_per_clk(probe, 1, False) * probe["sm_count"] * 2070.0 * 1e6  # explicit log grid
    cores = oracle.openmp_threads() or 1
    K = max(3, args.steps)
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    out = []

    def median_ms(fn, kernel_events=False, reps=None):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        call, kern = [], []
        for _ in range(reps or K):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            e1.record(stream)
            if kernel_events:
                gbkde.kde_set_kernel_events(e0, e1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            call.append(time.perf_counter() - t0)
            gbkde.kde_set_kernel_events()
            kern.append(e0.elapsed_time(e1) if kernel_events else 0.0)
        return 1e3 * statistics.median(call), statistics.median(kern)

    # n = 1,024 FP64 mixture
    n = 1024
    x = datagen.mixture_1d(n, seed=1)
    xd = torch.from_numpy(x).cuda()
    h = oracle.grid_log(0.01, 2.0, 64)
    grid, _keep = gbkde.make_grid(h=h)
    ws = gbkde.workspace(max(gbkde.kde_workspace_size(n, 1, 64), gbkde.kde_workspace_size(n, 1, 0)))
    P = n * (n - 1) // 2
    evals = P * (64 + 2)
    # n = 1,024 calls take about 0.1 ms: medians of 200 (host-side jitter of a few us per call)
    K1 = max(K, 200)
    sel_ms, _ = median_ms(lambda: (gbkde.kde_lscv(xd, grid, None, ws, stream), gbkde.kde_plugin(xd, None, ws, stream)),
                          reps=K1)
    # both selections as one replayed batch plan (one prologue, one graph launch)
    req, req_keep = gbkde.make_request(xd, gbkde.KDE_METHOD_LSCV | gbkde.KDE_METHOD_PLUGIN, grid)
    plan = gbkde.BatchPlan([req], keepalive=[req_keep])
    ws_plan = gbkde.workspace(plan.ws_bytes)
    plan_ms, _ = median_ms(lambda: plan.run(ws_plan, stream), reps=K1)
    plan_res = plan.run(ws_plan, stream)[0]
    sep_l = gbkde.kde_lscv(xd, grid, None, ws, stream)[0]
    sep_p = gbkde.kde_plugin(xd, None, ws, stream)
    plan_same = plan_res["h"] == sep_l["h"] and plan_res["h_plugin"] == sep_p["h"]
    _, kern_ms = median_ms(lambda: gbkde.kde_lscv(xd, grid, None, ws, stream), kernel_events=True, reps=K1)
    xh = torch.from_numpy(x).pin_memory().numpy()
    e2e_ms, _ = median_ms(lambda: (gbkde.kde_lscv_host(xh, grid, None, ws, stream),
                                   gbkde.kde_plugin_host(xh, None, ws, stream)), reps=K1)
    t0 = time.perf_counter()
    oracle.lscv_h(x, h)
    oracle.plugin(x)
    o_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.lscv_h(x, h, threads=1)
    oracle.plugin(x, threads=1)
    o1_s = time.perf_counter() - t0
    out.append({"config": "n=1024 FP64 mixture, 64-point LSCV on [0.01, 2] + plug-in", "evals": evals,
                "selection_ms": sel_ms, "evals_per_s": evals / (sel_ms * 1e-3),
                "selection_plan_ms": plan_ms, "plan_results_equal": plan_same,
                "lscv_kernel_ms": kern_ms, "lscv_kernel_evals_per_s": P * 64 / (kern_ms * 1e-3),
                "lscv_kernel_frac": P * 64 / (kern_ms * 1e-3) / peak, "e2e_ms": e2e_ms,
                "oracle_full_s": o_s, "oracle_evals_per_s": evals / o_s, "oracle_cores": cores,
                "oracle_single_thread_s": o1_s, "oracle_single_thread_evals_per_s": evals / o1_s})
    # d = 2, 3, 4, n = 16,384
    n = 16384
    P = n * (n - 1) // 2
    for d in (2, 3, 4):
        x = datagen.correlated_mixture(n, d, seed=3 + d)
        xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
        grid, _keep = gbkde.make_grid(n_h=128)  # default grid: 16 points per octave of 1/h^2
        peak_d = lscv_per_clk(probe, d, True) * probe["sm_count"] * 2070.0 * 1e6
        ws = gbkde.workspace(gbkde.kde_workspace_size(n, d, 128))
        sel_ms, kern_ms = median_ms(lambda: gbkde.kde_lscv(xd, grid, None, ws, stream), kernel_events=True)
        xh = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).pin_memory().numpy()
        e2e_ms, _ = median_ms(lambda: gbkde.kde_lscv_host(xh, grid, None, ws, stream))
        x64 = np.asarray(x, dtype=np.float32).astype(np.float64)
        hh = oracle.grid_default(n, d, 128)
        rows = 8 * cores
        t0 = time.perf_counter()
        oracle.lscv_sums(x64, hh, block=(0, rows, 0, n))
        o_s = time.perf_counter() - t0
        o_pairs = sum(n - 1 - i for i in range(rows))
        out.append({"config": f"d={d} n=16384 correlated mixture, 128-point LSCV over Z(h0)",
                    "evals": P * 128, "selection_ms": sel_ms, "evals_per_s": P * 128 / (sel_ms * 1e-3),
                    "lscv_kernel_ms": kern_ms, "lscv_kernel_evals_per_s": P * 128 / (kern_ms * 1e-3),
                    "lscv_kernel_frac": P * 128 / (kern_ms * 1e-3) / peak_d,
                    "lscv_roofline_evals_per_s": peak_d, "e2e_ms": e2e_ms,
                    "oracle_evals_per_s": o_pairs * 128 / o_s, "oracle_cores": cores,
                    "oracle_sample": f"rows 0..{rows - 1} of the pair triangle ({o_pairs} pairs, {o_s:.1f} s)"})
    # LSCV_H minimisation (Nelder-Mead over positive-definite H, Sec. 4.4.3)
    # of the same d = 2, 3, 4 sets from the normal-scale start
    for d in (2, 3, 4):
        x = datagen.correlated_mixture(n, d, seed=3 + d)
        xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
        p = d * (d + 1) // 2
        ws = gbkde.workspace(max(gbkde.kde_workspace_size(n, d, 1),
                                 gbkde.kde_lscv_H_workspace_size(n, d, max(4, p + 1))))
        gbkde.kde_lscv_H_minimize(xd, max_iter=20, ws=ws)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        H, g, evals = gbkde.kde_lscv_H_minimize(xd, max_iter=1000, ftol=1e-9, ws=ws)
        torch.cuda.synchronize()
        ms = 1e3 * (time.perf_counter() - t0)
        out.append({"config": f"d={d} n=16384 correlated mixture, LSCV_H Nelder-Mead minimisation",
                    "g_evaluations": evals, "ms": ms, "ms_per_g_evaluation": ms / max(1, evals),
                    "pair_evals_per_s": evals * P / (ms * 1e-3), "g_min": g,
                    "H": np.asarray(H).tolist()})
    clocks = sampler.stop()
    print(json.dumps({"workload": "configs", "peak_evals_per_s_2070mhz": peak, "results": out,
                      "clocks": clocks}), flush=True)
    return 0


def run_consumers(args):
    """Consumers of a selected bandwidth (Sec. 4.2, 4.3): the density estimate
    at query points (query x sample pairs, one exp2 each) and the range
    Count / Sum of one column (sample x range terms).  Per instance: the call
    end to end (perf_counter, results on the host), the pair kernel alone
    (CUDA events on the launching stream) and its ALU roofline."""
    import numpy as np
    import torch

    from paper_1505_01998_gb300 import datagen, gbkde

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    probe = gbkde.kde_probe_alu()
    K = max(1, args.steps)
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    out = []

    def timed(fn):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        call, kern = [], []
        for _ in range(K):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)  # torch creates the CUDA event at its first record
            e1.record(stream)
            gbkde.kde_set_kernel_events(e0, e1)
            t0 = time.perf_counter()
            fn()
            call.append(time.perf_counter() - t0)
            gbkde.kde_set_kernel_events()
            kern.append(e0.elapsed_time(e1))
        return 1e3 * statistics.median(call), statistics.median(kern)

    def alu_peak(fp32_per_eval, mufu_per_eval):
        per_clk = min(probe["mufu_ex2_per_clk_sm"] / mufu_per_eval,
                      probe["ffma_lanes_per_clk_sm"] / fp32_per_eval)
        return per_clk * probe["sm_count"] * 2070.0 * 1e6

    for d, n, m in ((1, 65536, 65536), (4, 65536, 16384), (16, 16384, 16384)):
        x = (datagen.skewed_column(n, seed=2) if d == 1 else datagen.correlated_mixture(n, d, seed=30 + d))
        xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
        S = np.atleast_2d(np.cov(x.astype(np.float64)))
        H = (0.25 if d > 1 else 0.01) * 0.5 * (S + S.T)
        g = datagen.rng(50 + d)
        lo, hi = x.min(axis=1), x.max(axis=1)
        q = (lo[:, None] + (hi - lo)[:, None] * g.uniform(size=(d, m))).astype(np.float32)
        if d == 1:
            q = np.linspace(lo[0], hi[0], m, dtype=np.float32)[None, :]
        qd = torch.from_numpy(np.ascontiguousarray(q)).cuda()
        ws = gbkde.workspace(gbkde.kde_eval_workspace_size(n, d, m))
        call_ms, kern_ms = timed(lambda: gbkde.kde_eval(xd, H, qd, ws, stream))
        evals = float(n) * m
        fp32 = 2 * d + 1  # per pair: d differences, d squared-distance FMAs, the running add
        peak = alu_peak(fp32, 1.0)
        out.append({"instance": f"kde_eval d={d} n={n} m={m}", "evals": evals,
                    "call_ms": call_ms, "kernel_ms": kern_ms,
                    "kernel_evals_per_s": evals / (kern_ms * 1e-3),
                    "call_evals_per_s": evals / (call_ms * 1e-3),
                    "roofline": {"bound": "alu", "peak_evals_per_s": peak,
                                 "frac": evals / (kern_ms * 1e-3) / peak,
                                 "basis": f"min(MUFU 1 ex2, FP32 {fp32} lanes) per pair at 2070 MHz"}})
    n, m = 1 << 24, 64
    x = datagen.skewed_column(n, seed=3)
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
    g = datagen.rng(60)
    lo = np.quantile(x[0][:: 64], g.uniform(0, 0.9, m))
    hi = lo + g.uniform(0, 1.0, m) * float(x.std())
    ws = gbkde.workspace(gbkde.kde_aqp_workspace_size(n, m))
    call_ms, kern_ms = timed(lambda: gbkde.kde_aqp(xd, 0.3, lo, hi, ws, stream))
    terms = float(n) * m
    out.append({"instance": f"kde_aqp n={n} ranges={m}", "terms": terms, "call_ms": call_ms,
                "kernel_ms": kern_ms, "kernel_terms_per_s": terms / (kern_ms * 1e-3),
                "call_terms_per_s": terms / (call_ms * 1e-3)})
    clocks = sampler.stop()
    print(json.dumps({"workload": "consumers", "instances": out, "clocks": clocks,
                      "alu_probe": probe}), flush=True)
    return 0


# ------------------------------------------------------------------ GPU leg

def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--n", type=int, default=N,
                    help="sample count (default 65536; smaller values only for profiling captures)")
    ap.add_argument("--workload", choices=("selection", "batch", "serve", "paper", "consumers", "configs"),
                    default="selection",
                    help="selection (default): the benchmark line; batch / serve: the batched and "
                         "served workloads, printed as their own JSON lines")
    ap.add_argument("--precision", choices=("kahan", "plain"), default="kahan",
                    help="per-thread summation of the pair kernels (selection workload)")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--autotune", action="store_true",
                    help="batch workload: tune the small-size buckets before planning")
    ap.add_argument("--serve-count", type=int, default=120)
    ap.add_argument("--serve-budget-gb", type=int, default=40)
    ap.add_argument("--serve-quantum", type=float, default=0.0,
                    help="work per scheduling step in direct-kernel evaluations (0 = the library default)")
    ap.add_argument("--rates", type=float, nargs="+", default=[10, 30, 100, 300, 1000, 2000])
    ap.add_argument("--serve-seeds", type=int, nargs="+", default=[5],
                    help="arrival seeds per rate (the serve workload reports median and range)")
    ap.add_argument("--rates-extra", type=float, nargs="+", default=[30, 100, 2000],
                    help="selection workload: serving rates of the line's serve object")
    ap.add_argument("--serve-count-extra", type=int, default=200)
    ap.add_argument("--serve-seeds-extra", type=int, nargs="+", default=[5, 6, 7])
    ap.add_argument("--shard", action="store_true",
                    help="selection workload: split one selection over the ranks (tile ranges + "
                         "NCCL all-reduce, strong scaling) instead of one replica per rank")
    ap.add_argument("--no-extras", action="store_true",
                    help="selection workload: skip the error, plain-precision, serving and batch "
                         "sub-measurements (profiling runs)")
    args = ap.parse_args()
    set_n(args.n)
    world, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, None, rank)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "paper":
        return run_paper(args)
    if args.workload == "consumers":
        return run_consumers(args)
    if args.workload == "configs":
        return run_configs(args)
    if args.shard:
        return run_shard(args, world, rank, local)
    return run_gpu(args, world, rank, local)


def kernel_event_pair(stream):
    """Two timing events recorded once on `stream`, so that torch treats them
    as recorded; kde_set_kernel_events then re-records them around a kernel."""
    import torch
    e = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    e[0].record(stream)
    e[1].record(stream)
    return e


def selection_errors(gbkde, xd, grid, opts, ws_l, ws_p):
    """Error of the selection left in the workspaces against the FP64 oracle
    over all pairs of the same samples (tests/golden/skewed65536_oracle.json,
    written by the oracle alone): g(h) at every grid point relative to
    max(|g|, its positive-term scale), S1 and S2 relative, the argmin, and the
    PLUGIN chain relative."""
    import numpy as np

    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "skewed65536_oracle.json")))
    r_l, g = gbkde.read_ws_result(ws_l, N_H)
    r_p, _ = gbkde.read_ws_result(ws_p)
    h = np.asarray(gold["h"])
    s_kk, s_k, g_ref = (np.asarray(gold[k]) for k in ("s_kk", "s_k", "g"))
    T = gbkde.kde_item_tiles(N, 1, N_H, opts)["lscv_tile"]
    s1, s2 = gbkde.kde_lscv_tile_sums(xd, h, 0, gbkde.kde_tile_count(N, T), opts)
    A = (4 * math.pi) ** -0.5 / gold["plugin"]["sigma"]
    scale = A * h ** -1.0 * (2.0 / N ** 2 * (s_kk + 2 ** 1.5 * s_k) + 1.0 / N)
    g_err = np.abs(g - g_ref) / np.maximum(np.abs(g_ref), scale)
    floor = pairs(N) * 2.0 ** -126
    rel = lambda a, b: abs(a - b) / abs(b)
    k_ref = int(gold["argmin"])
    return {"vs": "FP64 oracle over all 2.1e9 pairs of the same samples (tests/golden/skewed65536_oracle.json)",
            "tolerance": 1e-5,
            "lscv_g_max": float(g_err.max()),
            "lscv_s1_max_rel": float((np.abs(s1 - s_kk) / np.maximum(s_kk, floor)).max()),
            "lscv_s2_max_rel": float((np.abs(s2 - s_k) / np.maximum(s_k, floor)).max()),
            "lscv_argmin": int(r_l["argmin"]), "oracle_argmin": k_ref,
            "lscv_argmin_same": int(r_l["argmin"]) == k_ref,
            "lscv_h_rel": rel(r_l["h"], h[k_ref]),
            "psi6_rel": rel(r_p["psi6"], gold["plugin"]["psi6"]),
            "g2_rel": rel(r_p["g2"], gold["plugin"]["g2"]),
            "psi4_rel": rel(r_p["psi4"], gold["plugin"]["psi4"]),
            "plugin_h_rel": rel(r_p["h"], gold["plugin"]["h"])}


def selection_extras(args, xd, grid, opts, ws_l, ws_p, stream, flush, probe, sm_mhz):
    """Sub-measurements of the default line, outside its timed region: errors
    of the timed selection against the FP64 oracle, the same selection with
    plain FP32 per-thread sums (time and errors), the serving sweep and the
    512-dataset batch."""
    import torch

    from paper_1505_01998_gb300 import gbkde

    out = {"errors": selection_errors(gbkde, xd, grid, opts, ws_l, ws_p)}
    # plain FP32 sums: same kernels without compensation
    po = gbkde.make_opts(precision=gbkde.KDE_FP32_PLAIN)
    wl = gbkde.workspace(gbkde.kde_workspace_size(N, 1, N_H, po))
    wp = gbkde.workspace(gbkde.kde_workspace_size(N, 1, 0, po))
    for _ in range(2):
        gbkde.kde_lscv_async(xd, grid, po, wl, stream)
        gbkde.kde_plugin_async(xd, po, wp, stream)
    torch.cuda.synchronize()
    kms, sms = [], []
    for _ in range(5):
        flush.zero_()
        k0, k1 = kernel_event_pair(stream)
        e = [torch.cuda.Event(enable_timing=True), k0, k1, torch.cuda.Event(enable_timing=True)]
        e[0].record(stream)
        gbkde.kde_set_kernel_events(e[1], e[2])
        gbkde.kde_lscv_async(xd, grid, po, wl, stream)
        gbkde.kde_set_kernel_events()
        gbkde.kde_plugin_async(xd, po, wp, stream)
        e[3].record(stream)
        torch.cuda.synchronize()
        kms.append(e[1].elapsed_time(e[2]))
        sms.append(e[0].elapsed_time(e[3]))
    km = statistics.median(kms)
    out["plain"] = {"precision": "fp32 terms, plain fp32 per-thread sums, fp64 reductions",
                    "lscv_kernel_ms": km, "lscv_kernel_evals_per_s": EVALS_LSCV / (km * 1e-3),
                    "selection_ms": statistics.median(sms),
                    "selection_evals_per_s": EVALS_STEP / (statistics.median(sms) * 1e-3),
                    "errors": selection_errors(gbkde, xd, grid, po, wl, wp)}
    del wl, wp
    t0 = time.perf_counter()
    out["serve"] = serve_measure(args.rates_extra, args.serve_count_extra, args.serve_seeds_extra,
                                 args.serve_budget_gb, args.serve_quantum, repeat_from_rate=100.0)
    out["serve"]["wall_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    out["batch"] = batch_measure(args.batch_count, 2, 1)
    out["batch"]["wall_s"] = time.perf_counter() - t0
    return out


def run_shard(args, world, rank, local):
    """One selection (LSCV_h + PLUGIN of the n = 65,536 skewed column) split
    over the ranks: every rank evaluates a contiguous range of the pair
    tiles, then one NCCL all-reduce per all-pairs pass (2 n_h values for
    LSCV_h, one each for psi_6 and psi_4).  Strong scaling: the job is one
    selection whatever the rank count; value = its evaluations / the slowest
    rank's time per step (host clock between barriers: every step ends with
    host-side merges)."""
    import numpy as np
    import torch

    from paper_1505_01998_gb300 import datagen, gbkde
    from paper_1505_01998_gb300.shard import sharded_lscv, sharded_plugin

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    x = datagen.skewed_column(N, seed=SEED)
    xd = torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    h = gbkde.kde_default_grid(N, 1, N_H)

    def step():
        res_l, _ = sharded_lscv(xd, h)
        res_p = sharded_plugin(xd)
        return res_l, res_p

    W, K = max(3, args.warmup), args.steps
    for _ in range(W):
        res_l, res_p = step()
    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    t0 = time.perf_counter()
    for _ in range(K):
        res_l, res_p = step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    total_s = time.perf_counter() - t0
    clocks = sampler.stop()
    if dist:
        t = torch.tensor([total_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    ms = 1e3 * total_s / K
    line = {"metric": METRIC, "value": EVALS_STEP / (ms * 1e-3), "unit": UNIT, "n_gpus": world,
            "steps": K, "warmup": W, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD + ", one selection sharded over the ranks", "n": N, "d": 1,
                       "n_h": N_H, "evals_per_step": EVALS_STEP, "seed": SEED,
                       "parallelism": f"tile-range shards x{world}, NCCL all-reduce of 2 n_h + 2 FP64 values",
                       "timing": "host clock between barriers (steps end with host merges)"},
            "clocks": clocks,
            "result": {"lscv_argmin": res_l["argmin"], "lscv_h": res_l["h"], "plugin_h": res_p["h"]}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_gpu(args, world, rank, local):
    import numpy as np
    import torch

    from paper_1505_01998_gb300 import datagen, gbkde

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    x = datagen.skewed_column(N, seed=SEED + rank)
    xd = torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    grid, _keep = gbkde.make_grid(n_h=N_H)
    opts = gbkde.make_opts(precision=gbkde.KDE_FP32_PLAIN if args.precision == "plain" else gbkde.KDE_FP32_KAHAN)
    ws_l = gbkde.workspace(gbkde.kde_workspace_size(N, 1, N_H, opts), dev)
    ws_p = gbkde.workspace(gbkde.kde_workspace_size(N, 1, 0, opts), dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    probe = gbkde.kde_probe_alu()

    def step():
        gbkde.kde_lscv_async(xd, grid, opts, ws_l, stream)
        gbkde.kde_plugin_async(xd, opts, ws_p, stream)

    W, K = max(3, args.warmup), args.steps
    for _ in range(W):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    r_l, _ = gbkde.read_ws_result(ws_l, N_H)
    r_p, _ = gbkde.read_ws_result(ws_p)
    assert r_l["status"] == 0 and r_p["status"] == 0, (r_l, r_p)

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(K)]
    for e6 in ev:
        for e in e6:
            e.record(stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    for k in range(K):
        flush.zero_()  # 256 MiB write (> 129 MB L2) between steps, outside the step events
        e = ev[k]
        e[0].record(stream)
        gbkde.kde_set_kernel_events(e[2], e[3], e[4], e[5])
        step()
        e[1].record(stream)
    gbkde.kde_set_kernel_events()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    step_ms = [ev[k][0].elapsed_time(ev[k][1]) for k in range(K)]
    lscv_ms = statistics.mean(ev[k][2].elapsed_time(ev[k][3]) for k in range(K))
    psi_ms = statistics.mean(ev[k][4].elapsed_time(ev[k][5]) for k in range(K))
    total_ms = sum(step_ms)
    if dist:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / K
    value = EVALS_STEP * world / (ms_per_step * 1e-3)

    # ---- the same selection on the 256-point log grid over the closed interval
    # [h0/4, 4 h0] (not octave-shaped: the direct kernel), LSCV kernel timed alone
    h0 = (4.0 / (3.0 * N)) ** 0.2  # normal-scale h0 for d = 1, in units of sigma
    grid_c, _keep_c = gbkde.make_grid(n_h=N_H, h_min=h0 / 4.0, h_max=4.0 * h0)
    for _ in range(2):
        gbkde.kde_lscv_async(xd, grid_c, opts, ws_l, stream)
    torch.cuda.synchronize()
    closed_ms = []
    for k in range(max(3, K // 2)):
        flush.zero_()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        c1.record(stream)
        torch.cuda.synchronize()
        gbkde.kde_set_kernel_events(c0, c1)
        gbkde.kde_lscv_async(xd, grid_c, opts, ws_l, stream)
        gbkde.kde_set_kernel_events()
        torch.cuda.synchronize()
        closed_ms.append(c0.elapsed_time(c1))
    closed_kernel_ms = statistics.median(closed_ms)

    # ---- end to end: pinned host samples in, results out, through the public API
    x_pin = torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
    xh = x_pin.numpy()
    for _ in range(W):
        gbkde.kde_lscv_host(xh, grid, opts, ws_l, stream)
        gbkde.kde_plugin_host(xh, opts, ws_p, stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e2e_s = 0.0
    for _ in range(K):
        flush.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        gbkde.kde_lscv_host(xh, grid, opts, ws_l, stream)
        gbkde.kde_plugin_host(xh, opts, ws_p, stream)
        e2e_s += time.perf_counter() - t1
    if dist:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = EVALS_STEP * world * K / e2e_s
    h2d = 2 * N * 4
    # LSCV: one copy of the workspace span from the result to the end of g[n_h];
    # PLUGIN: the result struct
    r_off, g_off = gbkde.kde_ws_result_offset()
    d2h = (g_off + 8 * N_H - r_off) + ctypes.sizeof(gbkde.kde_result)

    # ---- roofline of the dominant kernel (all-pairs LSCV)
    sm_mhz = (clocks or {}).get("sm_mhz") or probe["sm_mhz"]
    per_clk = lscv_per_clk(probe, 1, True)  # the default 256-point grid: 32 points per octave
    peak = per_clk * probe["sm_count"] * sm_mhz * 1e6 / 1e9
    achieved = EVALS_LSCV / (lscv_ms * 1e-3) / 1e9
    peak_max = per_clk * probe["sm_count"] * 2070.0 * 1e6 / 1e9
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Geval/s",
                "frac": achieved / peak, "traffic": profiled_lscv_traffic(),
                "kernel": "k_lscv (all-pairs, all-bandwidths LSCV)",
                "kernel_ms": lscv_ms, "evals_per_launch": EVALS_LSCV,
                "peak_basis": (lscv_basis(probe, 1, True, sm_mhz) + " (median SM clock sampled during "
                               "the timed region); unit counts measured by kde_probe_alu"),
                "peak_at_max_clock": peak_max, "frac_at_max_clock": achieved / peak_max,
                "psi_kernel_ms": psi_ms,
                "psi_geval_s": pairs(N) / (psi_ms * 1e-3) / 1e9,
                "closed_grid": {
                    "grid": "256-point log grid over the closed [h0/4, 4 h0] (direct kernel: one ex2 per evaluation)",
                    "kernel_ms": closed_kernel_ms,
                    "geval_s": EVALS_LSCV / (closed_kernel_ms * 1e-3) / 1e9,
                    "peak": lscv_per_clk(probe, 1, False) * probe["sm_count"] * sm_mhz * 1e6 / 1e9,
                    "frac": EVALS_LSCV / (closed_kernel_ms * 1e-3) / 1e9
                    / (lscv_per_clk(probe, 1, False) * probe["sm_count"] * sm_mhz * 1e6 / 1e9)}}

    # ratio to the basis of one MUFU ex2 per evaluation (the direct kernel's
    # bound): above 1 on the default grid, whose octave shape lets most
    # exponentials be formed by squaring
    roofline["frac_vs_one_ex2_basis"] = achieved / (probe["mufu_ex2_per_clk_sm"] * probe["sm_count"] * sm_mhz * 1e6 / 1e9)
    # the bound of the octave kernel's earlier form (three FMUL2 scalings per 16
    # evaluations, 1.5 FMUL2/FADD2 lanes per evaluation): a fixed yardstick
    # across versions, since the exponent adds moved the instruction-mix bound
    fp32_3fmul = 1.0 / (1.5 / probe["fmul2_fadd2_lanes_per_clk_sm"] + 0.375 / probe["ffma2_lanes_per_clk_sm"]
                        + (2.0 / 16.0) / probe["ffma_lanes_per_clk_sm"])
    roofline["frac_vs_three_fmul2_mix"] = achieved / (
        min(probe["mufu_ex2_per_clk_sm"] / 0.375, fp32_3fmul) * probe["sm_count"] * sm_mhz * 1e6 / 1e9)

    extras = {}
    if rank == 0 and world == 1 and not args.no_extras and N == 65536:
        extras = selection_extras(args, xd, grid, opts, ws_l, ws_p, stream, flush, probe, sm_mhz)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N, "d": 1, "n_h": N_H,
                       "evals_per_step": EVALS_STEP, "seed": SEED,
                       "precision": ("fp32 terms, plain fp32 per-thread sums, fp64 reductions"
                                     if args.precision == "plain" else
                                     "fp32 terms, Kahan fp32 per-thread sums, fp64 reductions"),
                       "l2": "flushed between steps (256 MiB write outside the timed events)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": LAUNCHES_PER_STEP * K * world,  # all ranks
            "roofline": roofline, "clocks": clocks,
            "alu_probe": probe,
            "result": {"lscv_argmin": r_l["argmin"], "lscv_h": r_l["h"], "plugin_h": r_p["h"],
                       # the skewed column's g(h) still falls at h0/4, the lower end of Z(h0)
                       "lscv_min_at_lower_edge": bool(r_l["flags"] & gbkde.KDE_FLAG_MIN_AT_LOWER_EDGE)}}
    line.update(extras)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = oracle_sample(args.cpu_seconds)
        cb.pop("seconds")
        line["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
