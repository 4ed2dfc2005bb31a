#!/usr/bin/env python
"""Benchmark of the nested Monte Carlo hot path: path-steps/s on the 5-asset max-call.

One step = the whole hot path over one batch: for S0 in {90, 100, 110}, the Ibanez-Zapatero
fit (5 boundaries x J=1024 Korobov points per date, N1 = 1e5 inner paths per continuation
estimate, device Newton to |f| < 1e-6 or the x tolerance, FP64 quadratic regression, 8 fitted
dates) and the final pricing with 1e6 paths (plus the FP64 re-run of the pricing that states
the FP32 error).  value = inner + pricing path-steps actually simulated / device time.  The
Newton passes run in the cooperative form (one launch per date, --launch-mode); the JSON line
also times the fit of one option in all three launch forms on the same seeds (launch_forms).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun every rank runs its own replica of the step (independent options, different
seeds; no collective on the data path) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# before any CUDA context exists: hardware queues for the serving loop's per-request streams
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

from bap_workloads import IZParams, serving_stream, spec_max_call  # noqa: E402

S0S = (90.0, 100.0, 110.0)
J_FULL, N1_FULL, N_PRICE = 1024, 100_000, 1_000_000
METRIC = "nested-MC path-steps/s (5-asset max-call)"
WORKLOAD = "5-asset max-call Bermudan, I&Z, rho=0.3, J=1024 Korobov, N1=1e5, 9 dates, N=1e6"
# CPU sample of the same workload for the oracle (about 10-30 s of CPU work)
CPU_J, CPU_N1, CPU_NPRICE = 64, 4000, 100_000


def component_ops_per_path_step(d: int = 5) -> dict:
    """Algorithmic 32-bit lane operations of one path-step of the I&Z max-call path, counted
    by component: Philox4x32-10 at ceil(d/4) calls of 10 rounds x (2 mul-hi + 2 mul-lo + 2
    xor) plus the key schedule's bumps (80 per call), Box-Muller at 4 MUFU + 6 FP32 per pair,
    mixing and the log update at d(d+1)/2 + d FMA, the payoff's exp, the quadratic boundary at
    (d-1)d/2 + d FMA, and the counters, uniforms, argmax and stop test; in total, for d = 5,
    about 200 integer + 65 FP32 + 13 MUFU = 278 operations."""
    if d != 5:
        raise ValueError("the stated total is for d = 5")
    return {"int": 200, "fp32": 65, "mufu": 13, "total": 278}


def alg_ops_per_path_step(d: int = 5, degree: int = 2) -> dict:
    """A stricter count of the same path-step (the key schedule, which the kernel computes
    once per launch, and the loop's own bookkeeping left out): Philox4x32-10: ceil(d/4) calls x
    10 rounds x (2 wide multiplies + 4 xor); Box-Muller: ceil(d/2) pairs x (4 uniform ops + 4
    MUFU + 4 FP32); mixing d(d+1)/2 FMA; log-space step 2d; prices d exp2 (MUFU); argmax
    2(d-1); payoff 2; boundary: (d-1) selects + n_coef FMA + 1 compare."""
    s = d - 1
    n_coef = 1 + (s if degree >= 1 else 0) + (s * (s + 1) // 2 if degree >= 2 else 0)
    calls = (d + 3) // 4
    pairs = (d + 1) // 2
    ops = {
        "philox_int": calls * 10 * 6,
        "uniform_int": pairs * 4,
        "box_muller_fp32": pairs * 4,
        "mufu": pairs * 4 + d,
        "mix_fma": d * (d + 1) // 2,
        "step_fp32": 2 * d,
        "argmax_payoff": 2 * (d - 1) + 2,
        "rule": s + n_coef + 1,
    }
    ops["total"] = sum(ops.values())
    return ops


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def combine_ranks(elapsed_ms: float, steps: float, ws: int, device) -> tuple:
    """Whole-job numbers of a replica run: the slowest rank's timed span (max over ranks), the
    path-steps of all ranks (sum), and value = all steps / that span.  One process group call
    per reduction; with one rank nothing is exchanged."""
    if ws <= 1:
        return elapsed_ms, float(steps), float(steps) / (elapsed_ms / 1e3)
    import torch
    import torch.distributed as dist
    span = torch.tensor([elapsed_ms], dtype=torch.float64, device=device)
    total = torch.tensor([float(steps)], dtype=torch.float64, device=device)
    dist.all_reduce(span, op=dist.ReduceOp.MAX)
    dist.all_reduce(total, op=dist.ReduceOp.SUM)
    return float(span[0]), float(total[0]), float(total[0]) / (float(span[0]) / 1e3)


def run_reference(args) -> None:
    """The oracle (plain FP64 C + numpy) on the host cores, same metric and unit."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    spec = spec_max_call(5, 100.0, rho=0.3)
    params = IZParams(J=CPU_J, N1=CPU_N1, degree=2, seed=0)

    def one():
        t = time.perf_counter()
        rules, diag = oracle.iz_fit(spec, params, n_threads=cores)
        res = oracle.price(spec, rules, CPU_NPRICE, 1, n_threads=cores)
        el = time.perf_counter() - t
        return sum(d["steps"] for d in diag.values()) + res["path_steps"], el

    for _ in range(args.warmup):
        one()
    steps = secs = 0.0
    for _ in range(args.steps):
        s, e = one()
        steps += s
        secs += e
    value = steps / secs
    sample = (f"oracle I&Z fit of the 5-asset max-call (rho=0.3, S0=100, 9 dates) at J={CPU_J}, "
              f"N1={CPU_N1}, all 8 fitted dates, plus {CPU_NPRICE} pricing paths; FP64; OpenMP "
              f"over items; per step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "path-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (bounded CPU sample, see cpu_baseline)",
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "path-steps/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "path-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline() -> dict:
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    spec = spec_max_call(5, 100.0, rho=0.3)
    params = IZParams(J=CPU_J, N1=CPU_N1, degree=2, seed=0)
    t = time.perf_counter()
    rules, diag = oracle.iz_fit(spec, params, n_threads=cores)
    res = oracle.price(spec, rules, CPU_NPRICE, 1, n_threads=cores)
    el = time.perf_counter() - t
    steps = sum(d["steps"] for d in diag.values()) + res["path_steps"]
    # the same oracle on one thread, on a quarter of the items and a fifth of the pricing paths
    p1 = IZParams(J=CPU_J // 4, N1=CPU_N1, degree=2, seed=0)
    t = time.perf_counter()
    rules1, diag1 = oracle.iz_fit(spec, p1, n_threads=1)
    res1 = oracle.price(spec, rules1, CPU_NPRICE // 5, 1, n_threads=1)
    el1 = time.perf_counter() - t
    steps1 = sum(d["steps"] for d in diag1.values()) + res1["path_steps"]
    return {"value": steps / el, "unit": "path-steps/s", "cores": cores, "kind": "oracle",
            "sample": (f"I&Z fit of the 5-asset max-call (rho=0.3, S0=100, 9 dates) at "
                       f"J={CPU_J}, N1={CPU_N1}, 8 fitted dates + {CPU_NPRICE} pricing paths "
                       f"({steps} path-steps in {el:.1f} s); FP64 C with OpenMP over items"),
            "single_thread": {"value": steps1 / el1, "unit": "path-steps/s", "cores": 1,
                              "sample": (f"the same at J={p1.J}, N1={CPU_N1} + {CPU_NPRICE // 5} "
                                         f"pricing paths ({steps1} path-steps in {el1:.1f} s)")}}


def serving_bench(bap, n_req: int, max_inflight: int, budget: int) -> dict:
    """The mixed request stream (Poisson arrivals, mean 2 ms; d ~ U{1..10}; 4..50 dates; inner
    budget log-uniform 1e4..1e6; mixed payoffs; I&Z or CMC) replayed in real time through the
    server, then through the plain per-request form: the same direct calls one request at a
    time, one launch per Newton pass.  Latency = completion - arrival on the host clock."""
    reqs = serving_stream(n=n_req, seed=0)

    def summary(lat, span):
        lat = sorted(lat)
        return {"options_per_s": len(lat) / span, "p50_ms": 1e3 * lat[len(lat) // 2],
                "p99_ms": 1e3 * lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                "makespan_s": span}

    srv = bap.Server(budget, max_inflight)
    t0 = time.perf_counter()
    pending, served, lat = {}, {}, {}
    i = 0
    while i < len(reqs) or pending:
        now = time.perf_counter() - t0
        while i < len(reqs) and reqs[i].arrival_s <= now:
            r = reqs[i]
            pending[srv.submit(r.spec, r.params, r.n_paths, r.seed)] = i
            i += 1
        done = []
        for t, j in pending.items():
            out = srv.poll(t)
            if out is not None:
                served[j] = out[1]
                lat[j] = time.perf_counter() - t0 - reqs[j].arrival_s
                done.append(t)
        for t in done:
            del pending[t]
        if not done:
            time.sleep(0.0002)
    span_srv = time.perf_counter() - t0 - reqs[0].arrival_s
    stats = srv.stats()
    srv.close()

    t0 = time.perf_counter()
    plain, lat_p = {}, {}
    for j, r in enumerate(reqs):
        wait = r.arrival_s - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        o = bap.Option(r.spec)
        o.set_launch_mode(bap.LAUNCH_PLAIN)
        if r.method == "iz":
            o.fit_boundary(r.params)
        else:
            o.fit_classifier(r.params)
        plain[j] = o.price(r.n_paths, r.seed)
        o.close()
        lat_p[j] = time.perf_counter() - t0 - r.arrival_s
    span_plain = time.perf_counter() - t0 - reqs[0].arrival_s
    mismatches = sum(1 for j in range(len(reqs)) if served[j]["price"] != plain[j]["price"])
    steps = sum(v["fit_path_steps"] + v["path_steps"] for v in served.values())
    fp64 = [abs(v["fp64_delta"]) / v["se"] for v in served.values() if v["se"] > 0]
    return {"workload": f"{len(reqs)} requests, Poisson arrivals (mean 2 ms), d~U{{1..10}}, "
                        "4..50 dates, inner budget log-U[1e4,1e6], mixed payoffs, I&Z/CMC 50/50, "
                        "pricing 1e5 paths",
            "served": {**summary(list(lat.values()), span_srv), "max_inflight": max_inflight,
                       "peak_inflight": stats["peak_inflight"],
                       "server_thread_start_s": stats["start_ms"] / 1e3,
                       "server_thread_finish_s": stats["finish_ms"] / 1e3},
            "plain_per_request": summary(list(lat_p.values()), span_plain),
            "results_equal": mismatches == 0, "mismatches": mismatches,
            "fp64_delta_over_se": {"max": max(fp64) if fp64 else None,
                                   "median": statistics.median(fp64) if fp64 else None},
            "path_steps": steps}


LAUNCH_MODES = {"plain": 0, "graph": 1, "coop": 2}
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "path_kernel_5d_max_call.md")
PATH_SOURCES = [os.path.join(ROOT, "paper_0805_1827_gb300", "csrc", f)
                for f in ("bap_path.cuh", "bap_internal.cuh")]


def kernel_source_hash() -> str:
    """SHA-256 of the path kernel's sources with their comments and blank lines removed, so that
    an edit of comments alone leaves it unchanged."""
    import hashlib
    import re
    code = []
    for f in PATH_SOURCES:
        text = open(f, encoding="utf-8").read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        code += [line.rstrip() for line in text.splitlines() if line.strip()]
    return hashlib.sha256("\n".join(code).encode()).hexdigest()


def profiled_traffic():
    """DRAM bytes (read + write) per launch of the dominant kernel, the cooperative Newton
    launch, as ncu measured them on the full workload (profiles/path_kernel_5d_max_call.md);
    None when the kernel's code changed since that capture."""
    try:
        text = open(PROFILE_SUMMARY).read()
        src = kernel_source_hash()
    except OSError:
        return None
    fields = dict(line.split(":", 1) for line in text.splitlines()
                  if line.startswith(("source_sha256:", "dram_bytes_per_launch:")))
    if fields.get("source_sha256", "").strip() != src:
        return None
    try:
        return float(fields["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def continuation_fp64(bap, opt, params, n_sample: int = 64) -> dict:
    """The FP32 path's error of continuation estimates at the fit's boundary: for a sample of
    the last fit's boundary points of every date (start point S0 with the pivot asset at the
    point), the continuation sums under the fitted rules with the paths stepped in FP32 and in
    FP64 on the same counters (N1 paths each)."""
    import numpy as np
    from bap_workloads import PURPOSE_IZ
    spec = opt.spec
    rel = []
    for m in range(1, spec.n_dates):
        x, _, st = opt.fit_points(m)
        n_bnd = spec.d
        J = len(x) // n_bnd
        sel = np.linspace(0, len(x) - 1, n_sample // (spec.n_dates - 1) + 1).astype(int)
        sel = sel[st[sel] == 0]
        starts = np.zeros((len(sel), spec.d))
        piv = (sel // J).astype(np.int32)
        for k, i in enumerate(sel):
            starts[k, :] = spec.S0            # any positive start; the pivot carries the point
            starts[k, piv[k]] = x[i]
        g32, _ = opt.debug_continuation(m, PURPOSE_IZ, params.seed, sel, starts, params.N1, piv)
        g64, _ = opt.debug_continuation(m, PURPOSE_IZ, params.seed, sel, starts, params.N1, piv,
                                        fp64=True)
        c32, c64 = g32[:, 0] / params.N1, g64[:, 0] / params.N1
        rel += list(np.abs(c32 - c64) / np.maximum(np.abs(c64), 1e-12))
    rel = np.array(rel)
    return {"estimates": int(rel.size), "rel_diff_max": float(rel.max()),
            "rel_diff_median": float(np.median(rel)),
            "sample": (f"{rel.size} start points over all dates of the S0=100 fit: S0 with the "
                       "pivot asset at a fitted boundary point; N1 paths each, under the fitted "
                       "rules")}


def launch_forms(bap, params, stream) -> dict:
    """The I&Z fit of the S0=100 option in each launch form on the same seeds (identical fits
    and prices): one launch per Newton pass, one graph with conditional loops, one cooperative
    launch per date.  Device time of the fit from the library's own events."""
    out = {}
    for name, mode in LAUNCH_MODES.items():
        best = None
        for rep in range(2):
            o = bap.Option(spec_max_call(5, 100.0, rho=0.3), stream=stream.cuda_stream)
            o.set_launch_mode(mode)
            o.fit_boundary(params)
            r = o.price(100_000, 5)
            o.close()
            if best is None or r["fit_ms"] < best["fit_ms"]:
                best = r
        out[name] = {"fit_ms": best["fit_ms"], "kernel_launches": best["kernel_launches"],
                     "path_launches": best["path_launches"], "price": best["price"],
                     "se": best["se"], "fp64_delta": best["fp64_delta"]}
    prices = {v["price"] for v in out.values()}
    out["identical_prices"] = len(prices) == 1
    return out


def cmc_boost_forms(bap, stream) -> dict:
    """The CMC boosting forms side by side (one warp-per-feature block, a cluster of d+1 blocks,
    one 1024-thread block): first the serving-sized fit (5-asset max-call, J=1024 points, N2=200,
    200 stumps, 10 fitted dates; boosting time per date from the library's phase events), then
    the 7-asset basket put (J=4000, N2=2e4, 200 stumps, 9 fitted dates; device time of the whole
    fit).  Every form gives the same price."""
    from bap_workloads import CMCParams, spec_basket_put_7, spec_max_call
    names = {0: "one_block", 1: "cluster", 2: "warp_per_feature"}
    small = {}
    sspec = spec_max_call(5, 100.0, rho=0.3, n_dates=11, T=2.0)
    sparams = CMCParams(J=1024, N2=200, n_stumps=200, seed=1)
    for name, form in (("warp_per_feature", 2), ("cluster", 1), ("one_block", 0)):
        best = None
        for rep in range(2):
            o = bap.Option(sspec, stream=stream.cuda_stream)
            o.set_profiling(True)
            o.set_boost_form(form)
            o.fit_classifier(sparams)
            r = o.price(100_000, 5)
            o.close()
            if best is None or r["phase_ms"][2] < best["phase_ms"][2]:
                best = r
        small[name] = {"boost_ms_per_date": best["phase_ms"][2] / (sspec.n_dates - 1),
                       "fit_ms": best["fit_ms"], "price": best["price"], "se": best["se"],
                       "fp64_delta": best["fp64_delta"]}
    small["identical_prices"] = len({small[k]["price"] for k in names.values()}) == 1
    small["workload"] = "5-asset max-call, CMC, J=1024, N2=200, 200 stumps, 10 fitted dates"
    spec = spec_basket_put_7(0)
    params = CMCParams(J=4000, N2=20_000, n_stumps=200, seed=1)
    out = {"J1024": small}
    for name, form in (("warp_per_feature", 2), ("cluster", 1), ("one_block", 0)):
        best = None
        for rep in range(2):
            o = bap.Option(spec, stream=stream.cuda_stream)
            o.set_boost_form(form)
            o.fit_classifier(params)
            r = o.price(100_000, 5)
            r["form_ran"] = o.last_boost_form()
            o.close()
            if best is None or r["fit_ms"] < best["fit_ms"]:
                best = r
        out[name] = {"fit_ms": best["fit_ms"], "price": best["price"], "se": best["se"],
                     "fp64_delta": best["fp64_delta"], "form_ran": names[best["form_ran"]]}
    out["identical_prices"] = len({out[k]["price"] for k in names.values()}) == 1
    # LogitBoost (Section 3.2's alternative), 100 rounds = 200 vote stumps, on its cluster kernel
    lp = CMCParams(J=4000, N2=20_000, n_stumps=100, seed=1, boost=1)
    best = None
    for rep in range(2):
        o = bap.Option(spec, stream=stream.cuda_stream)
        o.fit_classifier(lp)
        r = o.price(100_000, 5)
        o.close()
        if best is None or r["fit_ms"] < best["fit_ms"]:
            best = r
    out["logitboost_cluster"] = {"fit_ms": best["fit_ms"], "price": best["price"], "se": best["se"],
                                 "fp64_delta": best["fp64_delta"], "rounds": 100}
    out["workload"] = "7-asset basket put, CMC, J=4000, N2=2e4, 200 stumps, 9 fitted dates"
    return out


def cmc_ops_per_path_step(d: int, n_stumps: int) -> int:
    """Algorithmic operations of one CMC label path-step of the d-asset basket put, counted by
    component: Philox4x32-10 ceil(d/4) calls x 80 (key schedule included), Box-Muller ceil(d/2)
    pairs x (4 MUFU + 6 FP32), mixing and the log update d(d+1)/2 + d, the basket payoff d exp
    + d FMA, and the stump rule (d+1) features x (ceil(log2(stumps per feature)) + 1) compares
    plus d+1 adds."""
    per_f = max(1, n_stumps // (d + 1))
    rule = (d + 1) * (math.ceil(math.log2(per_f)) + 1) + (d + 1)
    return ((d + 3) // 4) * 80 + ((d + 1) // 2) * 10 + d * (d + 1) // 2 + d + 2 * d + rule


def cmc_labels_7d(bap, stream, peak_ops: float) -> dict:
    """The CMC label paths of the 7-asset basket put (sigma_i ~ U[0.15, 0.35], seeded
    correlation, J = 4000 training points, N2 = 2e4 inner paths, 200 stumps, 9 fitted dates):
    inner path-steps per second of the [calc] phase (training points and label launches, CUDA
    events) and its fraction of the issue-slot peak."""
    from bap_workloads import CMCParams, spec_basket_put_7
    spec = spec_basket_put_7(0)
    params = CMCParams(J=4000, N2=20_000, n_stumps=200, seed=1)
    best = None
    for rep in range(2):
        o = bap.Option(spec, stream=stream.cuda_stream)
        o.set_profiling(True)
        o.fit_classifier(params)
        r = o.price(1_000_000, 5)
        o.close()
        if best is None or r["phase_ms"][1] < best["phase_ms"][1]:
            best = r
    rate = best["fit_path_steps"] / (best["phase_ms"][1] / 1e3)
    ops = cmc_ops_per_path_step(7, 200)
    return {"workload": "7-asset basket put, CMC, J=4000, N2=2e4, 200 stumps, 9 fitted dates",
            "path_steps_per_s": rate, "calc_ms": best["phase_ms"][1],
            "fit_path_steps": best["fit_path_steps"], "ops_per_path_step": ops,
            "frac": rate * ops / peak_ops, "fit_ms": best["fit_ms"],
            "boost_ms_per_date": best["phase_ms"][2] / (spec.n_dates - 1),
            "price": best["price"], "se": best["se"], "fp64_delta": best["fp64_delta"],
            "launch": bap.tuned_launch(7, "cmc", 0, 4000, 20_000)}


def paper_tables(bap) -> dict:
    """The paper's 3-asset max-call (Eq. 2 / Eq. 3) at its own settings: Table 1 (I&Z, J=128,
    N1=5e3), Table 2 (J sweep), Table 3 (N1 sweep), Table 4 (CMC, 5e3 points, N2=500, 200
    stumps), N=1e6 pricing paths; our price, SE and fit time beside the printed price, the
    printed binomial value and the printed minutes on 16 processors."""
    from bap_workloads import CMCParams
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_tables.json")))

    def run(s0, params):
        o = bap.Option(spec_max_call(3, float(s0)))
        if isinstance(params, IZParams):
            o.fit_boundary(params)
        else:
            o.fit_classifier(params)
        r = o.price(1_000_000, 2)
        o.close()
        return {"price": r["price"], "se": r["se"], "fp64_delta": r["fp64_delta"],
                "fit_ms": r["fit_ms"], "price_ms": r["price_ms"]}

    out = {"table1_iz": {}, "table2_iz_J": {}, "table3_iz_N1": {}, "table4_cmc": {}}
    for s0 in (90, 100, 110):
        g = gold["table1_iz"][str(s0)]
        out["table1_iz"][s0] = {**run(s0, IZParams(J=128, N1=5000, degree=2, seed=1)),
                                "paper_price": g["price"], "binomial": g["binomial"]}
    for J in (128, 256, 1024):
        g = gold["table2_iz_J"][str(J)]
        out["table2_iz_J"][J] = {**run(90, IZParams(J=J, N1=5000, degree=2, seed=1)),
                                 "paper_price": g["price"], "paper_minutes_16_procs": g["minutes_16_procs"]}
    for N1 in (5000, 10_000, 100_000):
        g = gold["table3_iz_N1"][str(N1)]
        out["table3_iz_N1"][N1] = {**run(90, IZParams(J=128, N1=N1, degree=2, seed=1)),
                                   "paper_price": g["price"], "paper_minutes_16_procs": g["minutes_16_procs"]}
    for s0 in (90, 100, 110):
        g = gold["table4_cmc"][str(s0)]
        out["table4_cmc"][s0] = {**run(s0, CMCParams(J=5000, N2=500, n_stumps=200, seed=1)),
                                 "paper_price": g["price"], "binomial": g["binomial"]}
    return out


def root_find_study(bap) -> dict:
    """Safeguarded Newton (from the bracket edge, and warm-started at the later date's fitted
    boundary) against the paper's literal fixed-point iteration (eps = 0.01) on the
    Table 1 workload (3-asset max-call, S0=90, J=128, N1=5e3, 8 fitted dates, max_iter 100):
    continuation evaluations per boundary point (mean, median, p90, max: the load imbalance
    among points), points without convergence, inner path-steps, fit time and price."""
    import numpy as np
    out = {}
    for name, fp, warm in (("newton", 0, 0), ("newton_warm_start", 0, 1), ("fixed_point", 1, 0)):
        spec = spec_max_call(3, 90.0)
        o = bap.Option(spec)
        p = IZParams(J=128, N1=5000, degree=2, seed=1, fixed_point=fp, fp_eps=0.01, max_iter=100,
                     warm_start=warm)
        o.fit_boundary(p)
        r = o.price(1_000_000, 2)
        its = np.concatenate([o.fit_points(m)[1] for m in range(1, spec.n_dates)])
        o.close()
        out[name] = {"evals_mean": float(its.mean()), "evals_p50": float(np.percentile(its, 50)),
                     "evals_p90": float(np.percentile(its, 90)), "evals_max": int(its.max()),
                     "points": int(its.size), "noconv": r["n_noconv"],
                     "fit_path_steps": r["fit_path_steps"], "fit_ms": r["fit_ms"],
                     "price": r["price"], "se": r["se"], "fp64_delta": r["fp64_delta"]}
    return out


def boundary_degree_study(bap) -> dict:
    """The I&Z boundary as a linear, quadratic or cubic polynomial (Section 2.2) on the Table 1
    workload (3-asset max-call, J=128, N1=5e3, N=1e6): price, SE and fit time per degree."""
    out = {}
    for s0 in (90, 100, 110):
        for deg in (1, 2, 3):
            o = bap.Option(spec_max_call(3, float(s0)))
            o.fit_boundary(IZParams(J=128, N1=5000, degree=deg, seed=1))
            r = o.price(1_000_000, 2)
            o.close()
            out[f"S0={s0},degree={deg}"] = {"price": r["price"], "se": r["se"],
                                            "fp64_delta": r["fp64_delta"], "fit_ms": r["fit_ms"]}
    return out


def run_ours(args) -> None:
    import torch
    import paper_0805_1827_gb300 as bap

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    props = torch.cuda.get_device_properties(dev)
    stream = torch.cuda.current_stream()
    J = args.J or J_FULL
    N1 = args.N1 or N1_FULL
    mode = LAUNCH_MODES[args.launch_mode]
    opts = [bap.Option(spec_max_call(5, s0, rho=0.3), stream=stream.cuda_stream) for s0 in S0S]
    for o in opts:
        o.set_launch_mode(mode)
        if args.paths_per_lane:
            o.set_paths_per_lane(args.paths_per_lane)
        if args.unit_paths:
            o.set_unit_paths(args.unit_paths)
    params = IZParams(J=J, N1=N1, degree=2, seed=1000 * rank + 1)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def step(seed_price: int):
        steps = launches = path_launches = 0
        kms = 0.0
        res = []
        for o in opts:
            o.fit_boundary(params)
            r = o.price(N_PRICE, seed_price)
            steps += r["fit_path_steps"] + r["path_steps"]
            launches += r["kernel_launches"]
            path_launches += r["path_launches"]
            kms += r["path_kernel_ms"]
            res.append(r)
        return steps, launches, path_launches, kms, res

    for i in range(args.warmup):
        step(7)
    for o in opts:
        o.set_profiling(True)
    sampler = ClockSampler(dev) if rank == 0 else None
    if sampler:
        sampler.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    times, tot_steps, tot_launch, tot_plaunch, tot_kms = [], 0, 0, 0, 0.0
    last = None
    for i in range(args.steps):
        flush.zero_()                       # evict L2 (129 MB) between timed steps
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        s, l, pl, kms, res = step(7)
        ev1.record(stream)
        torch.cuda.synchronize()
        times.append(ev0.elapsed_time(ev1))
        tot_steps += s
        tot_launch += l
        tot_plaunch += pl
        tot_kms += kms
        last = res
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    for o in opts:
        o.set_profiling(False)
    elapsed_ms = sum(times)
    elapsed_all, steps_all, value = combine_ranks(elapsed_ms, tot_steps, ws, dev)

    # end to end through the public API with host buffers: create (model H2D), fit, price (D2H)
    e2e_steps, e2e_secs = 0, 0.0
    h2d = d2h = 0
    for i in range(max(1, min(args.steps, 2))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s0 in S0S:
            spec = spec_max_call(5, s0, rho=0.3)
            o = bap.Option(spec)
            o.set_launch_mode(mode)
            o.fit_boundary(params)
            r = o.price(N_PRICE, 7)
            o.close()
            e2e_steps += r["fit_path_steps"] + r["path_steps"]
            if i == 0:
                h2d += 8 * (3 * spec.d + spec.d * spec.d)
                d2h += 8 * 16   # result struct plus the fit's and pricing's status reads
        e2e_secs += time.perf_counter() - t0
    e2e_value = e2e_steps / e2e_secs

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    cont64 = continuation_fp64(bap, opts[1], params)
    peaks0 = _peaks()
    peak_issue = props.multi_processor_count * 128 * float(peaks0.get("sm_max_mhz", 2070.0)) * 1e6
    cmc7 = cmc_labels_7d(bap, stream, peak_issue)
    forms = launch_forms(bap, params, stream) if args.launch_forms else None
    boost = cmc_boost_forms(bap, stream) if args.launch_forms else None
    tables = paper_tables(bap) if args.paper_tables else None
    rootfind = root_find_study(bap) if args.paper_tables else None
    degrees = boundary_degree_study(bap) if args.paper_tables else None

    ops = component_ops_per_path_step(5)
    strict = alg_ops_per_path_step(5, 2)
    peaks = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_ops = props.multi_processor_count * 128 * sm_max * 1e6    # lane-ops/s at max clock
    rate = tot_steps / (tot_kms / 1e3) if tot_kms > 0 else None    # path-steps/s in kernel
    achieved = rate * ops["total"] if rate else None
    roof = {"bound": "alu", "kernel": "path_kernel<5,IZ,float> (cooperative Newton launch)",
            "achieved": achieved / 1e12 if achieved else None,
            "peak": peak_ops / 1e12, "unit": "Tops/s",
            "frac": (achieved / peak_ops) if achieved else None,
            "traffic": profiled_traffic(),
            "traffic_basis": "ncu DRAM read+write bytes per cooperative Newton launch (full "
                             "workload, profiles/path_kernel_5d_max_call.md)",
            "ops_per_path_step": ops["total"],
            "ops_basis": "per d=5 path-step: Philox 2 calls x 80 (incl. key schedule), "
                         "Box-Muller 3 x (4 MUFU + 6 FP32), mixing 20, payoff 1 exp, boundary 15, "
                         "counters/uniforms/argmax/stop ~ 52: ~200 int + 65 FP32 + 13 MUFU",
            "frac_strict": (rate * strict["total"] / peak_ops) if rate else None,
            "ops_per_path_step_strict": strict["total"],
            "path_steps_per_s_in_kernel": rate,
            "peak_basis": (f"{props.multi_processor_count} SMs x 128 lane-ops/clk x {sm_max:.0f} "
                           "MHz (issue-slot peak; MEASURED_PEAKS sm_max_mhz)")}
    line = {
        "metric": METRIC, "value": value, "unit": "path-steps/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "options_per_step": len(S0S), "J": J, "N1": N1,
                   "N_price": N_PRICE, "l2": "flushed between timed steps (512 MiB write)",
                   "parallelism": f"replicas x{ws}"},
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": "path-steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": tot_launch,
        "roofline": roof,
        "launch_forms": forms,
        "cmc_boost_forms": boost,
        "paper_tables": tables,
        "root_find_study": rootfind,
        "boundary_degree_study": degrees,
        "continuation_fp64": cont64,
        "cmc_labels_7d": cmc7,
        "launch_config": {"5-asset I&Z fit": bap.tuned_launch(5, "iz", 2, 5 * J, N1),
                          "source": "autotuner table compiled into the library "
                                    "(paper_0805_1827_gb300/csrc/bap_tuning.inc)"},
        "prices": {f"S0={s0:g}": {"price": r["price"], "se": r["se"],
                                  "fp64_delta": r["fp64_delta"], "n_noconv": r["n_noconv"],
                                  "fit_path_steps": r["fit_path_steps"]}
                   for s0, r in zip(S0S, last)},
    }
    if args.serving > 0:
        line["serving"] = serving_bench(bap, args.serving, args.max_inflight, 64 << 30)
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving", type=int, default=512,
                    help="requests in the served-stream measurement (0: skip)")
    ap.add_argument("--max-inflight", type=int, default=32)
    ap.add_argument("--launch-mode", default="coop", choices=sorted(LAUNCH_MODES),
                    help="launch form of the I&Z Newton passes in the timed steps")
    ap.add_argument("--no-launch-forms", dest="launch_forms", action="store_false",
                    help="skip the side-by-side fit timings (I&Z launch forms, CMC boosting forms)")
    ap.add_argument("--no-paper-tables", dest="paper_tables", action="store_false",
                    help="skip the paper's Tables 1-4 workloads and the root-finding study")
    ap.add_argument("--paths-per-lane", type=int, default=0,
                    help="path slots per lane of the I&Z path kernels (0: the library's choice)")
    ap.add_argument("--unit-paths", type=int, default=0,
                    help="paths per warp unit of the fits (0: the library's choice)")
    ap.add_argument("--J", type=int, default=0, help="override J (testing only)")
    ap.add_argument("--N1", type=int, default=0, help="override N1 (testing only)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
