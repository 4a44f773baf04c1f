#!/usr/bin/env python3
"""Benchmark of the divide-and-combine copula estimator on GB300.

Headline workload: the batch of 4096 independent datasets (family uniform
over Gaussian / Frank / Gumbel, Kendall's tau ~ U[0.1, 0.8] mapped to theta,
n log-uniform in [1e3, 1e6], K = max(1, floor(n / 1e4)) equal subsets; about
6.1e8 FP32 pairs in 60,000 subsets; seeded synthetic data drawn from each
copula on the device).  One step = one CUDA-graph replay of the whole batched
fit: within-subset ranks (Eq. 12), per-rank transforms, the Newton passes
over the pseudo log-likelihood (Eq. 13), the sandwich variance and the Eq. 15
combine of every dataset.  The FP32-compensated path is the headline; the
FP64 path runs on the same inputs beside it.

Metric: pairs/s per likelihood pass = sum over subsets of (m x passes) / step
time, where passes is the number of Eq. 13 passes the subset's Newton driver
took (for the Gaussian family, solved from the sufficient statistics of one
pass, 1).  The step also ranks, tabulates, computes the variance and
combines, so this is a lower bound on the pass rate itself.

Extra keys: the Frank theta = 5, n = 1e6, K = 100 workload, the Gumbel
theta = 2, n = 1e8, K = 1000 lognormal-sized workload (the largest single
dataset), the Gaussian n = 1e4 latency case, the serving sweep, theta errors
against the FP64 oracle per workload and precision, and the oracle's own
stage timings on the host cores.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]
                  [--only mixed|frank_1m|gumbel_1e8|gauss_10k]

Under torchrun every rank fits its own replica of the workload (the method
is communication-free: replicas only), rank 0 prints one JSON line.
--impl reference times the FP64 CPU oracle's likelihood pass on this host's
cores on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pairs/s per likelihood pass & % roofline, FP32 vs FP64; serving fits/s, p50/p99"
WORKLOAD = "mixed_4096_datasets"
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2
FAMILY_NAMES = {0: "gaussian", 1: "frank", 2: "gumbel"}

# Algorithmic work per pair per likelihood pass in MUFU-class operations of
# each family, split by the unit class that issues them (ex2 for exp and
# expm1, lg2 for log, rcp for reciprocals), and per pair once per fit (the
# margin transforms):
#   Gaussian: no per-pass work (Newton runs on the sums A, B and m); two
#             normal quantiles per pair once (counted as one lg2 each).
#   Frank:    exp(-theta u), exp(-theta v), one expm1 for D; one reciprocal.
#   Gumbel:   x^theta, y^theta, w^(1/theta) (3 exp); log w, log(z + theta - 1)
#             (2 log); two reciprocals; log(-log u) of both margins once
#             (4 log).
# The sandwich variance costs two passes' worth (the per-point terms with
# their mixed partials).  HBM: one read of the FP32 pairs (8 B per pair);
# everything after lives in shared memory.
MUFU_PER_PASS = {0: (0.0, 0.0, 0.0), 1: (3.0, 0.0, 1.0), 2: (3.0, 2.0, 2.0)}   # (ex2, lg2, rcp)
MUFU_ONCE = {0: (0.0, 2.0, 0.0), 1: (0.0, 0.0, 0.0), 2: (0.0, 4.0, 0.0)}
VARIANCE_PASSES = 2.0
HBM_BYTES_PER_PAIR = 8.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--only", choices=["mixed", "frank_1m", "gumbel_1e8", "gauss_10k"], default=None,
                   help="run one workload alone (profiling); prints its own line")
    p.add_argument("--datasets", type=int, default=4096,
                   help="mixed only: datasets in the batch (smaller batches for profiling)")
    p.add_argument("--scale", type=float, default=1.0,
                   help="gumbel_1e8 only: n = 1e8 x scale pairs in 1000 x scale subsets (small profiling cases)")
    p.add_argument("--no-clocks", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--no-extras", action="store_true", help="headline workload only")
    p.add_argument("--no-oracle", action="store_true", help="skip the theta-error checks against the oracle")
    p.add_argument("--no-autotune", action="store_true", help="built-in block rule only (profiling runs)")
    p.add_argument("--blocks", default=None,
                   help="explicit F32C block table for every family instead of the autotuned one, "
                        "e.g. '10500:256,20480:512' (largest m : threads)")
    return p.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed loops run."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int, enabled: bool = True):
        self.device = device
        self.enabled = enabled
        self.proc = None
        self.path = None

    def start(self):
        if not self.enabled:
            return
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.12)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 10:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")

        load = [r for r in rows if num(r[4]) > 0] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in load for i in range(4) if r[6 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(num(r[1]) for r in load), "sm_max_mhz": max(num(r[2]) for r in rows),
                "samples": len(rows), "samples_under_load": len(load), "reasons": reasons}


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from
# the ncu captures summarised in profiles/, valid only for the kernel source
# they were taken on: the hash of those sources is recorded beside them and
# checked at run time (a changed kernel reports traffic null).
KERNEL_SOURCES = {
    "resident": ["resident.cu", "block_sort.cuh", "common.cuh", "families.cuh", "fit_common.cuh", "frank_series.h",
                 "internal.h"],
    "stream": ["stream.cu", "block_sort.cuh", "common.cuh", "families.cuh", "fit_common.cuh", "frank_series.h",
               "internal.h"],
}
CAPTURED_TRAFFIC = {
    # kernel: ({workload: bytes per step}, source hash at capture)
    # resident_kernel<float,u32,{256,512}> (autotuned tables) on the
    # 4096-dataset batch: 576.9 MB per step captured on the 512-dataset batch
    # of the same generator (ncu dram__bytes_read + dram__bytes_write),
    # scaled by pairs (611,948,340 / 70,224,133)
    "resident": ({WORKLOAD: 5028e6}, "b7007fafe7185408"),
    # stream_fit_kernel<float> on Gumbel n = 1e8, K = 1000: 7.414 GB read +
    # 3.137 GB written per launch, captured at full size (one ncu pass)
    "stream": ({"gumbel_1e8": 10551e6}, "4653dac98a03d11f"),
}


def kernel_source_hash(kernel):
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1609_05530_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def captured_traffic(kernel, workload):
    per_wl, sha = CAPTURED_TRAFFIC[kernel]
    if sha is None or sha != kernel_source_hash(kernel):
        return None
    return per_wl.get(workload)


def max_over_ranks(times, world, device):
    """Element-wise maximum of the per-rank timings (the job takes as long as
    its slowest rank); identity at one rank."""
    if world <= 1:
        return list(times)
    import torch
    import torch.distributed as dist
    t = torch.tensor(list(times), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def replica_throughput(world, units, steps, seconds):
    """Whole-job rate: every rank processes its own replica of `units` per step."""
    return world * units * steps / seconds


def passes_per_subset(fams, iters):
    """Eq. 13 passes per subset: the Newton driver's count, or 1 for the
    Gaussian family (its Newton iteration runs on the sums of one pass)."""
    it = np.asarray(iters, dtype=np.float64)
    return np.where(np.asarray(fams) == 0, 1.0, it)


def work_counts(m, fams, iters):
    """Algorithmic work of one fit of these subsets: (pair-passes, MUFU-class
    operations as (ex2, lg2, rcp) counts, HBM bytes)."""
    m = np.asarray(m, dtype=np.float64)
    fams = np.asarray(fams)
    it = np.asarray(iters, dtype=np.float64)
    pair_passes = float((m * passes_per_subset(fams, it)).sum())
    mufu = []
    for c in range(3):
        per_pass = np.array([MUFU_PER_PASS[int(f)][c] for f in fams])
        once = np.array([MUFU_ONCE[int(f)][c] for f in fams])
        mufu.append(float((m * (per_pass * (it + VARIANCE_PASSES) + once)).sum()))
    hbm = float(m.sum() * HBM_BYTES_PER_PAIR + m.shape[0] * 20.0)
    return pair_passes, tuple(mufu), hbm


def theta_errors(gpu_theta, gpu_status, o_theta, o_status, floor=0.05):
    """Errors of GPU estimates against the oracle's on the same subsets:
    relative |g - o| / |o| where |o| > floor, absolute where |o| <= floor
    (near independence a relative error is meaningless); only subsets with an
    estimate on both sides (status OK or BOUNDARY) are compared."""
    g = np.asarray(gpu_theta, dtype=np.float64)
    o = np.asarray(o_theta, dtype=np.float64)
    gs = np.asarray(gpu_status)
    os_ = np.asarray(o_status)
    ok = np.isin(os_, (0, 1)) & np.isin(gs, (0, 1)) & np.isfinite(o)
    big = ok & (np.abs(o) > floor)
    small = ok & ~big
    rel = np.abs(g[big] - o[big]) / np.abs(o[big])
    ab = np.abs(g[small] - o[small])
    return {"compared": int(ok.sum()), "status_mismatch": int((gs != os_).sum()),
            "max_rel": float(rel.max()) if rel.size else None,
            "median_rel": float(np.median(rel)) if rel.size else None,
            "near_zero": int(small.sum()), "max_abs_near_zero": float(ab.max()) if ab.size else None}


def combined_errors(gpu_comb, o_comb, floor=0.05):
    g = np.asarray(gpu_comb, dtype=np.float64)
    o = np.asarray(o_comb, dtype=np.float64)
    ok = np.isfinite(o) & np.isfinite(g)
    den = np.maximum(np.abs(o[ok]), floor)
    e = np.abs(g[ok] - o[ok]) / den
    return {"compared": int(ok.sum()), "max_rel": float(e.max()) if e.size else None}


def oracle_fits(u, v, off, fam, cores):
    import oracle
    return oracle.fit(fam, u, v, off, nthreads=cores)


def roofline(kind, work, kernel_ms, rates, peaks, peak_kind, clk, traffic, kernel_name, launches):
    """Roofline of the fused per-subset fit kernel: the slower of its HBM
    bytes at the measured copy bandwidth and its transcendental operations at
    the measured MUFU rates (ex2, lg2 and rcp timed apart: they issue at
    different rates) bounds it; achieved = that unit's work / the kernel time
    (CUDA events on the launching stream), peak = the rate the op mix allows."""
    pair_passes, (n_ex2, n_lg2, n_rcp), hbm = work
    secs = kernel_ms * 1e-3
    n_mufu = n_ex2 + n_lg2 + n_rcp
    t_mufu = n_ex2 / rates["mufu_ex2"] + n_lg2 / rates["mufu_lg2"] + n_rcp / rates["mufu_rcp"]
    mufu_peak = n_mufu / t_mufu if t_mufu > 0 else rates["mufu_ex2"]
    hbm_peak = peaks.get("hbm_gbs", 6800.0) * 1e9
    t_hbm = hbm / hbm_peak
    if t_mufu >= t_hbm:
        r = {"bound": "alu", "achieved": n_mufu / secs / 1e12, "peak": mufu_peak / 1e12, "unit": "Tops/s",
             "frac": t_mufu / secs,
             "peak_basis": "measured MUFU issue rates of this GPU (copula_measure_unit_rates, run inside this "
                           f"bench: ex2 {rates['mufu_ex2']:.3e}/s, lg2 {rates['mufu_lg2']:.3e}/s, rcp "
                           f"{rates['mufu_rcp']:.3e}/s) weighted by the op mix"}
    else:
        r = {"bound": "hbm", "achieved": hbm / secs / 1e9, "peak": hbm_peak / 1e9, "unit": "GB/s",
             "frac": t_hbm / secs, "peak_basis": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})"}
    r.update({
        "traffic": traffic, "traffic_unit": "bytes/step (all launches of the kernel)",
        "kernel": kernel_name, "launches_per_step": launches, "kernel_ms": kernel_ms,
        "work_per_step": {"pair_passes": pair_passes, "mufu_ex2": n_ex2, "mufu_lg2": n_lg2, "mufu_rcp": n_rcp,
                          "hbm_bytes": hbm},
        "hbm_frac": t_hbm / secs, "hbm_peak_kind": peak_kind, "mufu_frac": t_mufu / secs,
        "note": "work counted per pair per Eq. 13 pass (Frank 3 ex2 + 1 rcp, Gumbel 3 ex2 + 2 lg2 + 2 rcp, "
                "Gaussian none) plus the margin transforms once and the variance as two passes; 8 B of HBM per "
                "pair; the within-subset rank sort (shared memory, integer) is not counted as algorithmic work",
    })
    if clk:
        r["sm_mhz"] = clk.get("sm_mhz")
    return r


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def timed_replays(graph, steps, warm):
    import torch
    for _ in range(warm):
        graph.replay()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for s, e in ev:
        s.record()
        graph.replay()
        e.record()
    torch.cuda.synchronize()
    return [s.elapsed_time(e) / 1e3 for s, e in ev]


def bench_mixed(args, world, rank, rates, peaks, peak_kind, clocks, check_oracle):
    """The headline: 4096 datasets in one CUDA-graph replay per step."""
    import torch

    import paper_1609_05530_gb300 as cg
    from copula_synth import device as dsyn

    bt = dsyn.mixed_batch(B=args.datasets)
    dofs, soff, dss = bt["dataset_offsets"], bt["subset_offsets"], bt["dataset_subset_start"]
    n, B, S = int(dofs[-1]), len(dofs) - 1, int(dss[-1])
    m = np.diff(soff)
    sub_fam = np.repeat(bt["families"], np.diff(dss))
    from paper_1609_05530_gb300 import autotune
    ctxs = {p: cg.Context() for p in ("f32c", "f64")}
    t_tune = time.perf_counter()
    tables = {p: ({} if (args.no_autotune or args.blocks) else autotune.load_or_tune(p, "f32", ctx=ctxs[p]))
              for p in ("f32c", "f64")}
    if args.blocks:
        table = [tuple(int(x) for x in e.split(":")) for e in args.blocks.split(",")]
        cg.set_blocks(table, ctxs["f32c"])
        tables["f32c"] = {f: table for f in range(3)}
    t_tune = time.perf_counter() - t_tune
    ctx = ctxs["f32c"]
    res = {}
    # the same launch sequence with the built-in block rule, for comparison
    plan0 = cg.BatchPlan(bt["families"], dofs, soff, dss, precision="f32c", ctx=cg.Context())
    graph0 = plan0.capture(bt["u"], bt["v"])
    t_default = statistics.median(timed_replays(graph0, max(3, args.steps // 4), 2))
    del graph0
    plan0.close()
    clocks.start()
    for prec in ("f32c", "f64"):
        ctx = ctxs[prec]
        plan = cg.BatchPlan(bt["families"], dofs, soff, dss, precision=prec, ctx=ctx)
        graph = plan.capture(bt["u"], bt["v"])
        steps = args.steps if prec == "f32c" else max(3, args.steps // 4)
        warm = args.warmup if prec == "f32c" else max(3, args.warmup // 2)
        ts = timed_replays(graph, steps, warm)
        # launches and per-kernel time of the same launch sequence, outside the graph
        ctx.set_timing(True)
        kms = []
        for _ in range(max(3, steps // 4)):
            plan.run(bt["u"], bt["v"])
            kms.append(ctx.kernel_ms())
        ctx.set_timing(False)
        launches = ctx.launches()
        _, iters = plan.diagnostics()
        torch.cuda.synchronize()
        it = iters.cpu().numpy()
        res[prec] = {"times": ts, "kernel_ms": statistics.mean(kms), "launches": launches, "iters": it,
                     "theta": plan.theta.cpu().numpy(), "status": plan.status.cpu().numpy(),
                     "combined": plan.combined.cpu().numpy(), "steps": steps}
        del graph
        plan.close()
    clk = clocks.stop()
    t32 = sum(res["f32c"]["times"])
    t64 = sum(res["f64"]["times"])
    t32, t64 = max_over_ranks([t32, t64], world, "cuda")
    # pair-passes: the F32C path's Newton passes; the FP64 path's count also
    # holds its FP32 start search (as many passes as the F32C fit), counted
    # apart as FP32 work
    pp32 = float((m * passes_per_subset(sub_fam, res["f32c"]["iters"])).sum())
    it64 = np.maximum(res["f64"]["iters"] - np.where(sub_fam == 0, 0, res["f32c"]["iters"]), 0)
    pp64 = float((m * passes_per_subset(sub_fam, it64)).sum())
    steps32, steps64 = res["f32c"]["steps"], res["f64"]["steps"]
    value = replica_throughput(world, pp32, steps32, t32)
    val64 = replica_throughput(world, pp64, steps64, t64)
    work = work_counts(m, sub_fam, res["f32c"]["iters"])
    roof = roofline("mixed", work, res["f32c"]["kernel_ms"], rates, peaks, peak_kind, clk,
                    captured_traffic("resident", WORKLOAD), "resident_kernel<float,uint32_t,{512,256,128}>",
                    res["f32c"]["launches"])
    ctx = ctxs["f32c"]
    out = {"value": value, "ms_per_step": 1e3 * t32 / steps32, "steps": steps32, "clocks": clk,
           "autotune": {"tables": {p: {FAMILY_NAMES[f]: t for f, t in tables[p].items()} for p in tables},
                        "tune_or_load_s": t_tune, "default_blocks_ms_per_step": 1e3 * t_default,
                        "note": "block size per subset-size bucket and family, tuned on this GPU "
                                "(cached per GPU model, precision, storage, family)"},
           "gpu_launches": res["f32c"]["launches"] * steps32, "roofline": roof,
           "full_fit_pairs_per_s": world * n * steps32 / t32,
           "fits": {"datasets_per_s": world * B * steps32 / t32, "subsets_per_s": world * S * steps32 / t32},
           "passes_per_pair_f32c": pp32 / n, "kernel_ms_f32c": res["f32c"]["kernel_ms"],
           "fp64": {"value": val64, "unit": "pairs/s", "ms_per_step": 1e3 * t64 / steps64, "steps": steps64,
                    "kernel_ms": res["f64"]["kernel_ms"], "passes_per_pair": pp64 / n,
                    "full_fit_pairs_per_s": world * n * steps64 / t64,
                    "note": "FP64 passes only; the FP32 start search that precedes them is not counted"},
           "config": {"workload": WORKLOAD if B == 4096 else f"mixed_{B}_datasets", "datasets": B, "subsets": S,
                      "n": n,
                      "families": {FAMILY_NAMES[f]: int((bt["families"] == f).sum()) for f in range(3)},
                      "subset_m": {"min": int(m.min()), "median": int(np.median(m)), "max": int(m.max())},
                      "storage": "f32",
                      "precision": "f32c: FP32 per-point terms, compensated FP32 warp sums, FP64 across warps, "
                                   "FP64 Newton state, variance, combine",
                      "step": "one CUDA-graph replay of the batched fit: Eq. 12 ranks, tables, Newton passes "
                              "(Eq. 13), sandwich variance, Eq. 15 combine per dataset",
                      "value": "sum over subsets of m x Eq. 13 passes, per second of step time "
                               "(Gaussian: 1 pass, its Newton runs on the pass's sums)",
                      "l2": "inputs (4.9 GB) larger than L2; no flush", "parallelism": "1 GPU" if world == 1
                      else f"replicas x{world}"}}
    out["f32c_over_f64"] = (n * steps32 / t32) / (n * steps64 / t64)
    # end to end: host buffers through copula_fit_batch_host
    hu = torch.empty(n, dtype=torch.float32, pin_memory=True)
    hv = torch.empty(n, dtype=torch.float32, pin_memory=True)
    hu.copy_(bt["u"])
    hv.copy_(bt["v"])
    outs = (np.empty(S), np.empty(S), np.empty(S, dtype=np.int32), np.empty(B))
    o32 = cg.make_opts("f32c")
    cg.fit_batch_host(hu, hv, bt["families"], dofs, soff, dss, ctx=ctx, opts=o32, out=outs)
    e2e_steps = max(3, args.steps // 4)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        cg.fit_batch_host(hu, hv, bt["families"], dofs, soff, dss, ctx=ctx, opts=o32, out=outs)
    te = time.perf_counter() - t0
    (te,) = max_over_ranks([te], world, "cuda")
    out["e2e"] = {"value": world * pp32 * e2e_steps / te, "unit": "pairs/s",
                  "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": S * 20 + B * 8,
                  "ms_per_step": 1e3 * te / e2e_steps,
                  "call": "copula_fit_batch_host (pinned host u, v read by the fit kernel over the host link; "
                          "theta, var, status per subset and Eq. 15 per dataset copied back inside the call)"}
    del hu, hv
    if check_oracle and rank == 0:
        g = np.random.Generator(np.random.Philox(20260))
        order = g.permutation(B)
        pick, pairs = [], 0
        for b in order:  # whole datasets, about 3e6 pairs in all
            nb = int(dofs[b + 1] - dofs[b])
            if pairs + nb > 3_000_000:
                continue
            pick.append(int(b))
            pairs += nb
            if len(pick) >= 32:
                break
        cores = os.cpu_count() or 1
        errs = {p: {"th": [], "st": [], "oth": [], "ost": [], "comb": [], "ocomb": []} for p in ("f32c", "f64")}
        for b in sorted(pick):
            lo, hi = int(dofs[b]), int(dofs[b + 1])
            s0, s1 = int(dss[b]), int(dss[b + 1])
            u = bt["u"][lo:hi].cpu().numpy()
            v = bt["v"][lo:hi].cpu().numpy()
            o = oracle_fits(u, v, soff[s0:s1 + 1] - lo, int(bt["families"][b]), cores)
            for p in ("f32c", "f64"):
                e = errs[p]
                e["th"].append(res[p]["theta"][s0:s1])
                e["st"].append(res[p]["status"][s0:s1])
                e["oth"].append(o["theta"])
                e["ost"].append(o["status"])
                e["comb"].append(res[p]["combined"][b])
                e["ocomb"].append(o["combined"])
        out["theta_err_vs_oracle"] = {
            "sample": f"{len(pick)} whole datasets ({pairs} pairs, "
                      f"{sum(len(x) for x in errs['f32c']['th'])} subsets), seeded choice",
            **{p: {**theta_errors(np.concatenate(errs[p]["th"]), np.concatenate(errs[p]["st"]),
                                  np.concatenate(errs[p]["oth"]), np.concatenate(errs[p]["ost"])),
                   "combined": combined_errors(errs[p]["comb"], errs[p]["ocomb"])} for p in ("f32c", "f64")}}
    sample = dict(u=bt["u"], v=bt["v"], families=bt["families"], thetas=bt["thetas"], dofs=dofs, soff=soff, dss=dss)
    return out, sample


# Grid barriers of the streaming fit kernel after its Newton passes (the
# variance sweeps).
FIT_VARIANCE_BARRIERS = 5


def fit_phases(stamps, fit_ms, prec):
    """Spans (ms) of the streaming fit kernel's phases from its barrier
    timestamps: the table sweep, the Gaussian sums, the Newton passes (a chunk
    sweep and a step each; on the FP64 path the FP32 start search's passes
    come first, with three more barriers around them) and the variance
    sweeps up to the kernel's end."""
    t = np.concatenate([[0.0], np.asarray(stamps, dtype=np.float64)])
    nvar = FIT_VARIANCE_BARRIERS
    f64 = prec != "f32c"
    pre = 3 if f64 else 2  # FP64: the v-side table is gathered after its own barrier
    if len(t) < pre + nvar + 1:
        return None
    newton_end = len(t) - nvar - 1
    return {"tables": float(t[pre - 1]), "gaussian_sums": float(t[pre] - t[pre - 1]),
            "newton": float(t[newton_end] - t[pre]),
            "newton_passes": int((newton_end - pre - (3 if f64 else 0)) // 2),
            "variance": float(fit_ms - t[newton_end]),
            "variance_sweeps": [float(x) for x in np.diff(np.append(t[newton_end:], fit_ms))]}


def bench_frank_1m(args, check_oracle):
    """Frank theta = 5, n = 1e6 FP32, K = 100 equal subsets (8 MB of input)."""
    import torch

    import copula_synth as cs
    import paper_1609_05530_gb300 as cg

    d = cs.frank_1m(np.float32)
    u, v = torch.from_numpy(d.u).cuda(), torch.from_numpy(d.v).cuda()
    off = d.offsets
    m = np.diff(off)
    ctx = cg.Context()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    out = {}
    phases = None
    for prec in ("f32c", "f64"):
        o = cg.make_opts(prec)
        r, diag = cg.fit_ex(u, v, off, d.family, ctx=ctx, opts=o, phases=(prec == "f32c"))
        it = diag.iters.cpu().numpy()
        if prec == "f32c":
            ph = diag.phase_ns.cpu().numpy().astype(np.float64)
            dt = np.diff(ph, axis=1) / 1e3
            phases = {"ranks_us": float(dt[:, 0].mean()), "search_us": float(dt[:, 1].mean()),
                      "variance_us": float(dt[:, 2].mean()),
                      "subset_total_us": float((ph[:, 3] - ph[:, 0]).mean() / 1e3),
                      "kernel_span_us": float((ph[:, 3].max() - ph[:, 0].min()) / 1e3),
                      "note": "mean per-subset time of each phase from in-kernel global-timer stamps"}
        t_warm = time.perf_counter()
        while time.perf_counter() - t_warm < 0.3:  # clocks up before timing
            cg.fit(u, v, off, d.family, ctx=ctx, opts=o)
            torch.cuda.synchronize()
        steps = 50 if prec == "f32c" else 20
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        ctx.set_timing(True)
        kms = []
        for s, e in ev:
            flush.zero_()
            s.record()
            cg.fit(u, v, off, d.family, ctx=ctx, opts=o)
            e.record()
            kms.append(ctx.kernel_ms())
        ctx.set_timing(False)
        torch.cuda.synchronize()
        t = sum(s.elapsed_time(e) for s, e in ev) / 1e3
        out[prec] = {"t": t, "steps": steps, "kernel_ms": statistics.mean(kms), "iters": it,
                     "theta": r.theta.cpu().numpy(), "status": r.status.cpu().numpy(),
                     "combined": float(r.combined.item())}
    fam = np.full(len(m), d.family)
    pp32 = float((m * passes_per_subset(fam, out["f32c"]["iters"])).sum())
    pp64 = float((m * passes_per_subset(fam, out["f64"]["iters"] - out["f32c"]["iters"])).sum())
    line = {"workload": "frank_theta5_n1e6_K100_f32",
            "value": pp32 * out["f32c"]["steps"] / out["f32c"]["t"], "unit": "pairs/s",
            "ms_per_step": 1e3 * out["f32c"]["t"] / out["f32c"]["steps"], "kernel_ms": out["f32c"]["kernel_ms"],
            "full_fit_pairs_per_s": d.n * out["f32c"]["steps"] / out["f32c"]["t"],
            "passes_per_pair": pp32 / d.n,
            "fp64": {"value": pp64 * out["f64"]["steps"] / out["f64"]["t"],
                     "ms_per_step": 1e3 * out["f64"]["t"] / out["f64"]["steps"], "kernel_ms": out["f64"]["kernel_ms"]},
            "phases_f32c": phases,
            "l2": "flushed between timed steps (512 MB write, outside the timed span)"}
    line["f32c_over_f64"] = out["f64"]["t"] / out["f64"]["steps"] / (out["f32c"]["t"] / out["f32c"]["steps"])
    if check_oracle:
        o = oracle_fits(d.u, d.v, off, d.family, os.cpu_count() or 1)
        line["theta_err_vs_oracle"] = {
            "sample": "all 100 subsets",
            **{p: {**theta_errors(out[p]["theta"], out[p]["status"], o["theta"], o["status"]),
                   "combined": combined_errors([out[p]["combined"]], [o["combined"]])} for p in ("f32c", "f64")}}
    return line


def bench_rank_corr_inversion(check_oracle):
    """The rank-correlation inversion estimators (Section 2.3): per subset
    sample Kendall's tau and Spearman's rho (copula_rank_corr) on the Frank
    theta = 5, n = 1e6, K = 100 workload, then theta from each
    (copula_theta_from_rank_corr); and the inversion alone on 60,729 values
    (the subset count of the mixed batch) per family and map."""
    import torch

    import copula_synth as cs
    import paper_1609_05530_gb300 as cg

    d = cs.frank_1m(np.float32)
    u, v = torch.from_numpy(d.u).cuda(), torch.from_numpy(d.v).cuda()

    def timed(fn, reps=20):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            out = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, out

    ms_rc, (tau, rho) = timed(lambda: cg.rank_corr(u, v, d.offsets))
    ms_tau, (th_tau, st_tau) = timed(lambda: cg.theta_from_rank_corr(tau, cg.FRANK, "tau"))
    ms_rho, (th_rho, st_rho) = timed(lambda: cg.theta_from_rank_corr(rho, cg.FRANK, "rho"))
    out = {"workload": "frank_theta5_n1e6_K100_f32",
           "rank_corr_ms": ms_rc, "rank_corr_pairs_per_s": d.n / (ms_rc * 1e-3),
           "invert_tau_ms": ms_tau, "invert_rho_ms": ms_rho,
           "theta_tau_mean": float(th_tau.mean().item()), "theta_rho_mean": float(th_rho.mean().item())}
    g = np.random.Generator(np.random.Philox(31))
    many = {}
    for fam in (0, 1, 2):
        for which in ("tau", "rho"):
            r = torch.from_numpy(g.uniform(0.05, 0.85, 60_729)).cuda()
            ms, _ = timed(lambda: cg.theta_from_rank_corr(r, fam, which), reps=5)
            many[f"{FAMILY_NAMES[fam]}_{which}"] = {"ms": ms, "values_per_s": 60_729 / (ms * 1e-3)}
    out["invert_60729_values"] = many
    # streaming sizes: one subset of the largest streaming size (3,145,728
    # rows, sample-sort ranks, inversions chunk by chunk)
    from copula_synth import device as dsyn
    gg = torch.Generator(device="cuda")
    gg.manual_seed(6450)
    su, sv = dsyn.sample(cg.GUMBEL, 2.0, cg.MAX_SUBSET_STREAM, gg)
    su, sv = su.float(), sv.float()
    soff = np.array([0, cg.MAX_SUBSET_STREAM], dtype=np.int64)
    ms_s, _ = timed(lambda: cg.rank_corr(su, sv, soff), reps=5)
    out["rank_corr_streaming"] = {"m": cg.MAX_SUBSET_STREAM, "ms": ms_s,
                                  "pairs_per_s": cg.MAX_SUBSET_STREAM / (ms_s * 1e-3)}
    del su, sv
    if check_oracle:
        import oracle
        ot = np.array([oracle.theta_from_tau(1, float(t))[0] for t in tau.cpu().numpy()])
        e = np.abs(th_tau.cpu().numpy() - ot) / np.maximum(np.abs(ot), 0.05)
        out["theta_tau_err_vs_oracle"] = {"max_rel": float(e.max()), "subsets": int(e.shape[0]),
                                          "status_equal": bool(np.all(st_tau.cpu().numpy() == 0))}
    return out


PAPER_BOUNDS = {0: (0.002, 4e-6), 1: (0.008, 7e-5), 2: (0.008, 9e-5)}   # |bias|, MSE (Section 3.2)
PAPER_DIST_BOUND = 0.0013                                                 # relative L1, L2 (Section 3.2)
SIM_THETA = {0: 0.3, 1: 5.0, 2: 5.0}                                      # Section 2.5
SIM_DELTA = {0: 0.0, 1: 0.0, 2: 1e-6}


def bench_simulation_study(check_oracle, S=50):
    """The paper's simulation study (Sections 2.5-2.6) on the GPU: for each
    family at the paper's parameter, N in {5e4, 1e5, 2e5} and M in {10, 20,
    100}: S replicates drawn on the device, the M-subset fits (Eq. 16 per
    replicate) and the full-data fits in batched calls, then Eq. 17-20 by
    copula_simulation_summary; the estimated bias, MSE and relative L1 / L2
    distances against the bounds Section 3.2 reports.  The Gumbel
    distances are taken over [1e-6, 1 - 1e-6]^2 (its squared density is not
    integrable at (1, 1))."""
    import torch

    import copula_synth as cs
    import paper_1609_05530_gb300 as cg
    from copula_synth import device as dsyn

    ctx = cg.Context()
    rows = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gpu_ms = 0.0
    for fam in (0, 1, 2):
        th = SIM_THETA[fam]
        for N in (50_000, 100_000, 200_000):
            g = torch.Generator(device="cuda")
            us, vs = [], []
            for s_ in range(S):
                g.manual_seed(1605600 + 1000 * fam + N // 1000 + 7919 * s_)
                u, v = dsyn.sample(fam, th, N, g)
                us.append(u.float())
                vs.append(v.float())
            u, v = torch.cat(us), torch.cat(vs)
            del us, vs
            dofs = np.arange(S + 1, dtype=np.int64) * N
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            full = cg.fit_batch(u, v, [fam] * S, dofs, dofs, np.arange(S + 1, dtype=np.int64), "f32c", ctx=ctx)
            for M in (10, 20, 100):
                sub = np.concatenate([[0]] + [cs.equal_offsets(N, M)[1:] + s_ * N for s_ in range(S)]).astype(np.int64)
                r = cg.fit_batch(u, v, [fam] * S, dofs, sub, np.arange(S + 1, dtype=np.int64) * M, "f32c", ctx=ctx)
                summ = cg.simulation_summary(fam, r.combined, full.theta, SIM_DELTA[fam])
                rows.append((fam, N, M, summ, r.combined.clone(), full.theta.clone()))
            e1.record()
            torch.cuda.synchronize()
            gpu_ms += e0.elapsed_time(e1)
    wall = time.perf_counter() - t0
    out = []
    ok_all = True
    for fam, N, M, summ, comb, fullth in rows:
        d = dict(zip(cg.SIM_SUMMARY, summ.cpu().numpy().tolist()))
        bb, mb = PAPER_BOUNDS[fam]
        within = abs(d["bias"]) < bb and d["mse"] < mb and d["d1_relative"] < PAPER_DIST_BOUND and \
            d["d2_relative"] < PAPER_DIST_BOUND
        ok_all &= within
        row = {"family": FAMILY_NAMES[fam], "theta": SIM_THETA[fam], "N": N, "M": M,
               "theta_combined_sim": d["theta_combined_sim"], "theta_full_sim": d["theta_full_sim"],
               "bias": d["bias"], "mse": d["mse"], "d1_relative": d["d1_relative"], "d2_relative": d["d2_relative"],
               "within_paper_bounds": bool(within)}
        out.append(row)
    res = {"S": S, "configs": len(out), "fits": len(out) * S + 9 * S,
           "gpu_ms": gpu_ms, "wall_s": wall, "all_within_paper_bounds": bool(ok_all),
           "bounds": "Section 3.2: |bias| < 0.002 (Gaussian) / 0.008 (Frank, Gumbel); MSE < 4e-6 / 7e-5 / 9e-5; "
                     "relative L1 and L2 < 0.0013",
           "precision": "f32c fits; summaries and distances in FP64",
           "rows": out}
    if check_oracle:
        import oracle
        # the summary arithmetic of every configuration against the oracle's,
        # on the GPU's own estimates
        worst = 0.0
        for (fam, N, M, summ, comb, fullth), row in zip(rows, out):
            if M != 100:
                continue
            ref = oracle.simulation_summary(comb.cpu().numpy(), fullth.cpu().numpy())
            d1, d2 = oracle.relative_distances(fam, ref["theta_full_sim"], ref["theta_combined_sim"], SIM_DELTA[fam])
            for a, b in ((row["mse"], ref["mse"]), (row["d1_relative"], d1), (row["d2_relative"], d2)):
                worst = max(worst, abs(a - b) / max(abs(b), 1e-300))
        res["summary_rel_err_vs_oracle"] = worst
        res["summary_check"] = "MSE, Eq. 19, Eq. 20 of the 9 M = 100 configurations by the oracle's arithmetic " \
                               "and quadrature on the GPU's estimates"
    return res


def bench_gauss_10k(args, check_oracle):
    """Gaussian rho = 0.5, n = 1e4 FP64 storage, K = 10 (latency-bound)."""
    import torch

    import copula_synth as cs
    import paper_1609_05530_gb300 as cg

    d = cs.gaussian_10k(np.float64, K=10)
    u, v = torch.from_numpy(d.u).cuda(), torch.from_numpy(d.v).cuda()
    ctx = cg.Context()
    out = {}
    for prec in ("f32c", "f64"):
        o = cg.make_opts(prec, "equal")
        for _ in range(10):
            r = cg.fit(u, v, d.offsets, d.family, ctx=ctx, opts=o)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(100):
            r = cg.fit(u, v, d.offsets, d.family, ctx=ctx, opts=o)
        e1.record()
        torch.cuda.synchronize()
        out[prec] = {"us_per_fit": e0.elapsed_time(e1) * 10.0, "theta": r.theta.cpu().numpy(),
                     "status": r.status.cpu().numpy(), "combined": float(r.combined.item())}
    line = {"workload": "gaussian_rho0.5_n1e4_K10_f64", "us_per_fit_f32c": out["f32c"]["us_per_fit"],
            "us_per_fit_f64": out["f64"]["us_per_fit"], "combine": "equal weights"}
    if check_oracle:
        import oracle
        o = oracle.fit(d.family, d.u, d.v, d.offsets, weight=oracle.W_EQUAL, nthreads=os.cpu_count() or 1)
        line["theta_err_vs_oracle"] = {
            p: {**theta_errors(out[p]["theta"], out[p]["status"], o["theta"], o["status"]),
                "combined": combined_errors([out[p]["combined"]], [o["combined"]])} for p in ("f32c", "f64")}
    return line


def bench_gumbel_1e8(args, check_oracle, rates=None, peaks=None, peak_kind=None, clocks=None, steps=None):
    """Gumbel theta = 2, n = 1e8 FP32 pairs, K = 1000 lognormal(1)-sized
    subsets: 875 of them (98% of the pairs) above the single-block limit take
    the streaming path.  Inputs (800 MB) are larger than L2."""
    import torch

    import paper_1609_05530_gb300 as cg
    from copula_synth import device as dsyn

    u, v, off = dsyn.gumbel_lognormal(n=int(round(1e8 * args.scale)), K=max(1, int(round(1000 * args.scale))))
    n, K = int(off[-1]), len(off) - 1
    m = np.diff(off)
    ctx = cg.Context()
    out = {}
    for prec in ("f32c", "f64"):
        o = cg.make_opts(prec)
        st = steps or 10
        st = st if prec == "f32c" else max(3, st // 3)
        r, diag = cg.fit_ex(u, v, off, cg.GUMBEL, ctx=ctx, opts=o)
        it = diag.iters.cpu().numpy()
        for _ in range(2):
            cg.fit(u, v, off, cg.GUMBEL, ctx=ctx, opts=o)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(st):
            r = cg.fit(u, v, off, cg.GUMBEL, ctx=ctx, opts=o)
        ev[1].record()
        torch.cuda.synchronize()
        t = ev[0].elapsed_time(ev[1]) / 1e3
        ctx.set_timing(True)
        spans, total = [], []
        for _ in range(3):
            cg.fit(u, v, off, cg.GUMBEL, ctx=ctx, opts=o)
            total.append(ctx.kernel_ms())
            spans.append(ctx.stage_ms())
        stamps = ctx.stream_stamps() / 1e6  # barrier releases of the last call's fit kernel (ms)
        ctx.set_timing(False)
        sp = np.mean(np.array(spans), axis=0)
        out[prec] = {"t": t, "steps": st, "iters": it, "kernel_span_ms": float(np.mean(total)),
                     "stages_ms": {"shared_memory_subsets_and_setup": float(np.mean(total) - sp.sum()),
                                   "ranks_u": float(sp[0]), "ranks_v": float(sp[1]), "pi": float(sp[2]),
                                   "fit_kernel": float(sp[3])},
                     "fit_phases_ms": fit_phases(stamps, float(spans[-1][3]), prec),
                     "theta": r.theta.cpu().numpy(), "status": r.status.cpu().numpy(),
                     "combined": float(r.combined.item())}
    fam = np.full(K, cg.GUMBEL)
    pp32 = float((m * out["f32c"]["iters"]).sum())
    pp64 = float((m * np.maximum(out["f64"]["iters"] - out["f32c"]["iters"], 0)).sum())
    f = out["f32c"]
    big = m > cg.MAX_SUBSET
    nb = float(m[big].sum())
    itb = f["iters"][big].astype(np.float64)
    # algorithmic HBM bytes of the streaming fit kernel: the margin tables of
    # both coordinates written once (8 B/pair), read once per Newton pass and
    # twice for the variance (8 B/pair each)
    algo = {"ranks_u": 8.0 * nb, "ranks_v": 8.0 * nb,
            "fit_kernel": 8.0 * nb + 8.0 * float((m[big] * (itb + 2.0)).sum())}
    st_ms = f["stages_ms"]
    dom = max(algo, key=lambda k: st_ms[k])
    hbm = (peaks or {}).get("hbm_gbs", 6800.0)
    achieved = algo[dom] / (st_ms[dom] * 1e-3) / 1e9
    line = {"workload": "gumbel_theta2_n1e8_K1000_lognormal" if args.scale == 1.0
            else f"gumbel_theta2_n{n}_K{K}_lognormal",
            "n": n, "K": K, "streaming_subsets": int(big.sum()), "largest_subset": int(m.max()),
            "value": pp32 * f["steps"] / f["t"], "unit": "pairs/s", "ms_per_step": 1e3 * f["t"] / f["steps"],
            "full_fit_pairs_per_s": n * f["steps"] / f["t"], "passes_per_pair": pp32 / n,
            "stages_ms_f32c": st_ms, "fit_phases_ms_f32c": f["fit_phases_ms"],
            "kernel_span_ms_f32c": f["kernel_span_ms"],
            "fp64": {"value": pp64 * out["f64"]["steps"] / out["f64"]["t"],
                     "ms_per_step": 1e3 * out["f64"]["t"] / out["f64"]["steps"],
                     "stages_ms": out["f64"]["stages_ms"]},
            "f32c_over_f64": (out["f64"]["t"] / out["f64"]["steps"]) / (f["t"] / f["steps"]),
            "roofline_streaming": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                                   "frac": achieved / hbm, "algorithmic_bytes": algo[dom],
                                   "traffic": captured_traffic("stream", "gumbel_1e8") if args.scale == 1.0 else None},
            "l2": "inputs (800 MB) larger than L2"}
    if check_oracle:
        # the three smallest streaming subsets and three shared-memory ones
        g = np.random.Generator(np.random.Philox(20261))
        sm_idx = np.flatnonzero(~big)
        st_idx = np.flatnonzero(big)
        pick = list(st_idx[np.argsort(m[st_idx])[:3]]) + list(g.choice(sm_idx, size=min(3, sm_idx.size),
                                                                         replace=False))
        cores = os.cpu_count() or 1
        o_th, o_st = [], []
        for k in pick:
            lo, hi = int(off[k]), int(off[k + 1])
            o = oracle_fits(u[lo:hi].cpu().numpy(), v[lo:hi].cpu().numpy(), np.array([0, hi - lo]), cg.GUMBEL,
                            cores)
            o_th.append(o["theta"][0])
            o_st.append(o["status"][0])
        line["theta_err_vs_oracle"] = {
            "sample": f"subsets {sorted(int(k) for k in pick)} (m = {sorted(int(m[k]) for k in pick)})",
            **{p: theta_errors(out[p]["theta"][pick], out[p]["status"][pick], o_th, o_st) for p in ("f32c", "f64")}}
    return line


# ---------------------------------------------------------------------------
# the oracle on the host cores
# ---------------------------------------------------------------------------

def oracle_sample(sample, target_pairs, seed):
    """Whole subsets of the mixed batch, in seeded random order, up to
    target_pairs: [(family, theta, u, v)] as host arrays."""
    g = np.random.Generator(np.random.Philox(seed))
    soff, dss = sample["soff"], sample["dss"]
    S = len(soff) - 1
    sub_ds = np.repeat(np.arange(len(dss) - 1), np.diff(dss))
    out, pairs = [], 0
    for k in g.permutation(S):
        lo, hi = int(soff[k]), int(soff[k + 1])
        if pairs + (hi - lo) > target_pairs and out:
            break
        b = int(sub_ds[k])
        out.append((int(sample["families"][b]), float(sample["thetas"][b]), sample["u"][lo:hi].cpu().numpy(),
                    sample["v"][lo:hi].cpu().numpy()))
        pairs += hi - lo
    return out, pairs


def oracle_stages(subs, threads):
    """Time the oracle's stages over the subsets with `threads` host threads
    (one subset per task): ranks of both columns (Eq. 12), the per-point
    margin transforms, one Eq. 13 pass, and the full fit (grid-certified
    Newton, sandwich variance)."""
    import oracle
    pairs = sum(s[2].shape[0] for s in subs)

    def ranks(s):
        off = np.array([0, s[2].shape[0]], dtype=np.int64)
        return oracle.ranks(s[2], off), oracle.ranks(s[3], off)

    def run(fn, items):
        t0 = time.perf_counter()
        if threads == 1:
            r = [fn(x) for x in items]
        else:
            with ThreadPoolExecutor(threads) as ex:
                r = list(ex.map(fn, items))
        return r, time.perf_counter() - t0

    rk, t_rank = run(ranks, subs)
    built, t_xf = run(lambda a: oracle.Subset(a[0][0], a[1][0], a[1][1]), list(zip(subs, rk)))
    _, t_pass = run(lambda a: a[0].sums(a[1][1]), list(zip(built, subs)))
    for b in built:
        b.close()

    def fit(s):
        return oracle.fit(s[0], s[2], s[3], np.array([0, s[2].shape[0]], dtype=np.int64), nthreads=1)

    _, t_fit = run(fit, subs)
    return {"pairs": pairs, "subsets": len(subs), "rank_pairs_per_s": pairs / t_rank,
            "transform_pairs_per_s": pairs / t_xf, "pass_pairs_per_s": pairs / t_pass,
            "fit_pairs_per_s": pairs / t_fit, "fits_per_s": len(subs) / t_fit}


def cpu_baseline(sample):
    """The oracle as it stands, on bounded samples of the headline workload:
    single-threaded and on all host cores, stage by stage."""
    cores = os.cpu_count() or 1
    one, p1 = oracle_sample(sample, 120_000, 7)
    allc, pa = oracle_sample(sample, 120_000 * cores, 8)
    st1 = oracle_stages(one, 1)
    sta = oracle_stages(allc, cores)
    return {"value": sta["pass_pairs_per_s"], "unit": "pairs/s", "cores": cores, "kind": "oracle",
            "sample": f"single thread: {st1['subsets']} whole subsets ({p1} pairs); all cores: {sta['subsets']} "
                      f"whole subsets ({pa} pairs), seeded random choice from {WORKLOAD}; value = one Eq. 13 pass "
                      "(transforms prebuilt) on all cores",
            "single_thread": st1, "all_cores": sta}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import torch

    import oracle
    from copula_synth import device as dsyn
    cores = os.cpu_count() or 1
    on_gpu = torch.cuda.is_available()
    bt = dsyn.mixed_batch(B=4096) if on_gpu else dsyn.mixed_batch(B=64, device="cpu")
    workload = WORKLOAD if on_gpu else "mixed_64_datasets (drawn on the host: no GPU here)"
    sample = dict(u=bt["u"], v=bt["v"], families=bt["families"], thetas=bt["thetas"],
                  dofs=bt["dataset_offsets"], soff=bt["subset_offsets"], dss=bt["dataset_subset_start"])
    subs, pairs = oracle_sample(sample, 400_000 * cores, 9)
    off = [np.array([0, s[2].shape[0]], dtype=np.int64) for s in subs]
    built = [oracle.Subset(s[0], oracle.ranks(s[2], o), oracle.ranks(s[3], o)) for s, o in zip(subs, off)]

    def one_pass():
        t0 = time.perf_counter()
        with ThreadPoolExecutor(cores) as ex:
            list(ex.map(lambda a: a[0].sums(a[1][1]), zip(built, subs)))
        return time.perf_counter() - t0

    for _ in range(args.warmup):
        one_pass()
    tot = sum(one_pass() for _ in range(args.steps))
    for b in built:
        b.close()
    value = pairs * args.steps / tot
    line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": workload, "step": f"one Eq. 13 likelihood pass of the FP64 oracle over "
                                                     f"{len(subs)} whole subsets ({pairs} pairs) on {cores} "
                                                     f"host threads, transforms prebuilt"},
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                             "sample": f"{len(subs)} whole subsets ({pairs} pairs) of {workload}, seeded choice"},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# serving: Poisson arrivals of fit requests (family uniform over the three,
# Kendall tau ~ U[0.1, 0.8], n log-uniform in [1e4, 1e7] FP32 pairs, K = n/1e4)
# against the continuous-batching server under a 64 GB HBM budget
# ---------------------------------------------------------------------------

def serving_bench(pool_size=48, rates=(500, 1000, 2000, 4000, 8000), seconds=3.0, seed=1605535, solo_rounds=3):
    import torch

    import copula_synth as cs
    import paper_1609_05530_gb300 as cg
    from copula_synth import device as dsyn

    g = np.random.Generator(np.random.Philox(seed))
    pool = []
    tg = torch.Generator(device="cuda")
    for i in range(pool_size):
        fam = int(g.integers(0, 3))
        th = cs.theta_of_tau(fam, float(g.uniform(0.1, 0.8)))
        n = int(np.exp(g.uniform(np.log(1e4), np.log(1e7))))
        tg.manual_seed(seed + i)
        u, v = dsyn.sample(fam, th, n, tg)
        hu = torch.empty(n, dtype=torch.float32, pin_memory=True)
        hv = torch.empty(n, dtype=torch.float32, pin_memory=True)
        hu.copy_(u.float())
        hv.copy_(v.float())
        pool.append((fam, hu.numpy(), hv.numpy(), cs.equal_offsets(n, max(1, n // 10_000))))
        del u, v
    torch.cuda.synchronize()
    srv = cg.Server(64 << 30, max_slots=64, streams=4)
    for fam, u, v, off in pool[:4]:
        srv.wait(srv.submit(u, v, off, fam), 60)
    srv.reset_stats()
    solo, solo_n = [], []
    for _ in range(solo_rounds):
        for fam, u, v, off in pool:
            solo.append(srv.wait(srv.submit(u, v, off, fam), 60)["latency_s"])
            solo_n.append(int(u.shape[0]))
    slowest = np.argsort(solo)[-4:][::-1]
    unloaded = {"p50_ms": 1e3 * float(np.percentile(solo, 50)), "p99_ms": 1e3 * float(np.percentile(solo, 99)),
                "requests": len(solo),
                "slowest": [{"n": solo_n[i], "ms": round(1e3 * solo[i], 3)} for i in slowest],
                "largest_n_ms": round(1e3 * float(np.median([solo[i] for i in range(len(solo))
                                                             if solo_n[i] == max(solo_n)])), 3)}
    sweep = []
    for rate in rates:
        srv.reset_stats()
        tickets = []
        t_end = time.perf_counter() + seconds
        t_next = time.perf_counter()
        i = 0
        while True:
            now = time.perf_counter()
            if now >= t_end:
                break
            if now < t_next:
                time.sleep(min(t_next - now, 0.001))
                continue
            fam, u, v, off = pool[i % pool_size]
            tickets.append(srv.submit(u, v, off, fam))
            i += 1
            t_next += g.exponential(1.0 / rate)
        for t in tickets:
            srv.wait(t, 120)
        st = srv.stats()
        sweep.append({"offered_fits_per_s": rate, "fits_per_s": st["fits_per_s"], "p50_ms": 1e3 * st["p50_s"],
                      "p99_ms": 1e3 * st["p99_s"], "mean_batch": st["mean_batch"], "requests": len(tickets)})
    srv.close()
    ok = [r for r in sweep if r["p99_ms"] <= 2 * unloaded["p99_ms"]]
    best = max(ok, key=lambda r: r["offered_fits_per_s"]) if ok else None
    return {"workload": "Poisson arrivals; family uniform, tau ~ U[0.1,0.8], n log-uniform [1e4,1e7] FP32, "
                        f"K = n/1e4; pool of {pool_size} seeded requests; 64 GB arena, 64 slots, 4 streams",
            "unloaded": unloaded, "sweep": sweep,
            "stated_rate": best["offered_fits_per_s"] if best else None,
            "fits_per_s": best["fits_per_s"] if best else None,
            "p50_ms": best["p50_ms"] if best else None, "p99_ms": best["p99_ms"] if best else None,
            "rule": "highest offered rate whose p99 stays within 2x the unloaded p99"}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1609_05530_gb300 as cg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    check = not args.no_oracle and rank == 0 and world == 1
    peaks, peak_kind = measured_peaks()
    rates = cg.measure_unit_rates()
    clocks = ClockSampler(local, enabled=not args.no_clocks)

    if args.only in ("frank_1m", "gauss_10k", "gumbel_1e8"):
        fn = {"frank_1m": bench_frank_1m, "gauss_10k": bench_gauss_10k, "gumbel_1e8": bench_gumbel_1e8}[args.only]
        line = fn(args, check) if args.only != "gumbel_1e8" else fn(args, check, rates, peaks, peak_kind,
                                                                    clocks, args.steps)
        line["unit_rates"] = rates
        if rank == 0:
            print(json.dumps(line, default=float), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return 0

    head, sample = bench_mixed(args, world, rank, rates, peaks, peak_kind, clocks, check)
    if args.only == "mixed":
        if rank == 0:
            print(json.dumps({k: v for k, v in head.items()}, default=float), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return 0
    if rank != 0:
        dist.destroy_process_group()
        return 0
    line = {"metric": METRIC, "value": head["value"], "unit": "pairs/s", "n_gpus": world, "steps": head["steps"],
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": head["config"], "gpu_launches": head["gpu_launches"], "e2e": head["e2e"],
            "roofline": head["roofline"], "fp64": head["fp64"], "f32c_over_f64": head["f32c_over_f64"],
            "full_fit_pairs_per_s": head["full_fit_pairs_per_s"], "fits": head["fits"],
            "passes_per_pair_f32c": head["passes_per_pair_f32c"], "kernel_ms_f32c": head["kernel_ms_f32c"],
            "unit_rates": {k: v for k, v in rates.items()}, "unit_rates_unit": "results/s, whole GPU (measured)",
            "autotune": head["autotune"]}
    if head.get("clocks") is not None:
        line["clocks"] = head["clocks"]
    if "theta_err_vs_oracle" in head:
        line["theta_err_vs_oracle"] = head["theta_err_vs_oracle"]
    if not args.no_extras and world == 1:
        line["frank_1m"] = bench_frank_1m(args, check)
        line["gumbel_1e8"] = bench_gumbel_1e8(args, check, rates, peaks, peak_kind, clocks)
        line["gauss_10k"] = bench_gauss_10k(args, check)
        line["rank_corr_inversion"] = bench_rank_corr_inversion(check)
        line["simulation_study"] = bench_simulation_study(check)
    if not args.no_serving and world == 1:
        line["serving"] = serving_bench()
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(sample)
    print(json.dumps(line, default=float), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
