#!/usr/bin/env python3
"""Benchmark of the divide-and-combine copula estimator on GB300.

Workload: Frank copula theta = 5, n = 1,000,000 pairs stored FP32, K = 100
equal subsets of 10,000 (seeded synthetic data drawn from the copula by
conditional inversion).  One step = one complete fit through the C ABI:
within-subset ranks (Eq. 12), per-rank transforms, the Newton passes over the
pseudo log-likelihood (Eq. 13), the sandwich variance and the Eq. 15 combine.
The FP32-compensated path is the headline; the FP64 path runs on the same
inputs beside it.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]

Under torchrun every rank fits its own replica of the workload (the method
is communication-free), rank 0 prints one JSON line.  --impl reference times
the FP64 CPU oracle on this host's cores on bounded samples of the same
workload.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pairs/s per likelihood pass & % roofline, FP32 vs FP64; serving fits/s, p50/p99"
WORKLOAD = "frank_theta5_n1e6_K100_f32"
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-clocks", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--workload", choices=["frank_1m", "gauss_10k", "mixed_4096", "gumbel_1e8"], default="frank_1m")
    p.add_argument("--scale", type=float, default=1.0,
                   help="gumbel_1e8 only: n = 1e8 x scale pairs in 1000 x scale subsets (small profiling cases)")
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
    # kernel: (bytes per launch on the bench workload, source hash at capture)
    # resident_kernel<float,u32,512>, Frank n=1e6, K=100: 8.13 MB read, 0 written
    "resident": (8127744, "531f48d6c368d560"),
    # stream_fit_kernel<float>, Gumbel n=1e8, K=1000: 2.368 GB captured on the
    # n=2e7, K=200 case, scaled by streaming pairs (98,390,930 / 19,642,180)
    "stream": (11864180067, "a59f1a4b790877c8"),
}


def kernel_source_hash(kernel):
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1609_05530_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def captured_traffic(kernel):
    nbytes, sha = CAPTURED_TRAFFIC[kernel]
    if nbytes is None or sha != kernel_source_hash(kernel):
        return None
    return nbytes


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


def replica_throughput(world, n, steps, seconds):
    """Whole-job pairs/s: every rank fits its own n-pair replica per step."""
    return world * n * steps / seconds


def workload(name="frank_1m"):
    import copula_synth as cs
    if name == "gauss_10k":
        return cs.gaussian_10k(np.float64, K=10)
    return cs.frank_1m(np.float32)


# ---------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle on this host's cores
# ---------------------------------------------------------------------------

def oracle_sample(d, subsets, nthreads):
    import oracle
    lo, hi = int(d.offsets[0]), int(d.offsets[subsets])
    off = d.offsets[: subsets + 1] - lo
    t0 = time.perf_counter()
    oracle.fit(d.family, d.u[lo:hi], d.v[lo:hi], off, nthreads=nthreads)
    return hi - lo, time.perf_counter() - t0


def cpu_baseline(d, budget_s=20.0):
    """The oracle as it stands on the host cores, on a bounded sample of the
    workload (whole subsets, one per thread per round)."""
    cores = os.cpu_count() or 1
    sub = min(d.K, cores)
    pairs, dt = oracle_sample(d, sub, cores)
    rounds = max(1, min(d.K // sub, int(budget_s / max(dt, 1e-3))))
    tot_p, tot_t = 0, 0.0
    for r in range(rounds):
        p, t = oracle_sample(d, sub, cores)
        tot_p += p
        tot_t += t
    return {"value": tot_p / tot_t, "unit": "pairs/s", "cores": cores, "kind": "oracle",
            "sample": f"{rounds} round(s) of the first {sub} subsets ({sub * 10_000} pairs) of {WORKLOAD}, "
                      f"one subset per thread, full fit (ranks, grid-certified Newton, sandwich variance, combine)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    d = workload()
    cores = os.cpu_count() or 1
    budget = 150.0
    # size each step so that warmup + steps fit the budget
    p1, t1 = oracle_sample(d, 1, 1)
    per_step = budget / max(1, args.steps + args.warmup)
    sub = int(max(1, min(d.K, math.floor(per_step / max(t1, 1e-4)) * cores)))
    sub = max(1, min(d.K, sub))
    for _ in range(args.warmup):
        oracle_sample(d, sub, cores)
    tot_p, tot_t = 0, 0.0
    for _ in range(args.steps):
        p, t = oracle_sample(d, sub, cores)
        tot_p += p
        tot_t += t
    value = tot_p / tot_t
    line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "step": f"oracle fit of the first {sub} subsets"},
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                             "sample": f"first {sub} of {d.K} subsets per step"},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


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

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    d = workload(args.workload)
    fam = d.family
    u = torch.from_numpy(d.u).cuda()
    v = torch.from_numpy(d.v).cuda()
    off = d.offsets
    n = d.n
    ctx = cg.Context()
    o32 = cg.make_opts("f32c")
    o64 = cg.make_opts("f64")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    # passes per fit (Newton iterations are data-dependent; the count is fixed for fixed inputs)
    _, diag32 = cg.fit_ex(u, v, off, fam, ctx=ctx, opts=o32, phases=True)
    _, diag64 = cg.fit_ex(u, v, off, fam, ctx=ctx, opts=o64)
    m = np.diff(off)
    it32, it64 = diag32.iters.cpu().numpy(), diag64.iters.cpu().numpy()
    pair_passes32 = float((m * it32).sum())
    # the FP64 path's count includes its FP32 start search, the same passes
    # as the F32C fit of the same subset; the rest are FP64 passes
    pair_passes64 = float((m * (it64 - it32)).sum())
    ph = diag32.phase_ns.cpu().numpy().astype(np.float64)

    def timed_loop(opts, steps, warm):
        for _ in range(warm):
            cg.fit(u, v, off, fam, ctx=ctx, opts=opts)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        barrier()
        for k in range(steps):
            flush.zero_()
            starts[k].record()
            cg.fit(u, v, off, fam, ctx=ctx, opts=opts)
            ends[k].record()
        barrier()
        return sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / 1e3

    def kernel_loop(opts, steps):
        ctx.set_timing(True)
        ks = []
        for _ in range(steps):
            flush.zero_()
            cg.fit(u, v, off, fam, ctx=ctx, opts=opts)
            ks.append(ctx.kernel_ms())
        ctx.set_timing(False)
        return ks

    clocks = ClockSampler(local, enabled=not args.no_clocks)
    clocks.start()
    t32 = timed_loop(o32, args.steps, args.warmup)
    launches = ctx.launches()
    steps64 = max(10, args.steps // 10)
    t64 = timed_loop(o64, steps64, max(3, args.warmup // 4))
    kms32 = kernel_loop(o32, max(20, args.steps // 5))
    kms64 = kernel_loop(o64, max(10, steps64 // 2))

    # end to end through the host-buffer C entry point (the inputs cross the
    # host link and the results come back inside the call)
    hu = torch.from_numpy(d.u).pin_memory()
    hv = torch.from_numpy(d.v).pin_memory()
    outs = (np.empty(d.K), np.empty(d.K), np.empty(d.K, dtype=np.int32), np.empty(1))
    e2e_steps = max(10, args.steps // 10)
    for _ in range(3):
        cg.fit_host(hu, hv, off, fam, ctx=ctx, opts=o32, out=outs)
    te = 0.0
    for _ in range(e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cg.fit_host(hu, hv, off, fam, ctx=ctx, opts=o32, out=outs)
        te += time.perf_counter() - t0
    clk = clocks.stop()

    # max over ranks (each rank fits its own replica: no data-path collective)
    t32, t64, te = max_over_ranks([t32, t64, te], world, "cuda")
    if rank != 0:
        dist.destroy_process_group()
        return 0

    value = replica_throughput(world, n, args.steps, t32)
    search_rate = None
    if ph is not None and ph.size and d.K <= 152:
        search_us = float(np.mean(ph[:, 2] - ph[:, 1])) / 1e3
        search_rate = world * pair_passes32 / (search_us * 1e-6) if search_us > 0 else None
    val64 = world * n * steps64 / t64
    kms32_mean = statistics.mean(kms32)
    kms64_mean = statistics.mean(kms64)
    peaks, peak_kind = measured_peaks()
    roof = roofline(d, diag32, kms32_mean, clk, peaks, peak_kind)
    line = {
        "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t32 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": d.name if args.workload != "frank_1m" else WORKLOAD,
                   "family": {0: "gaussian", 1: "frank", 2: "gumbel"}[fam], "theta": d.theta, "n": n, "K": d.K,
                   "storage": "f64" if d.u.dtype == np.float64 else "f32",
                   "precision": "f32c: FP32 per-point terms, compensated FP32 warp sums, FP64 across warps, "
                                "FP64 Newton state, variance combine",
                   "step": "one complete fit per step: Eq. 12 ranks, tables, Newton passes (Eq. 13), sandwich "
                           "variance, Eq. 15 combine",
                   "value": "pairs fitted per second (n / step time)",
                   "l2": "flushed between timed steps (512 MB write, outside the timed span)",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "likelihood_pass": {
            "f32c_pairs_per_s": world * pair_passes32 * args.steps / t32,
            "f64_pairs_per_s": world * pair_passes64 * steps64 / t64,
            "passes_per_fit_f32c": pair_passes32 / n, "passes_per_fit_f64": pair_passes64 / n,
            "f64_start_search_passes_per_fit_f32": pair_passes32 / n,
            "note": "pair-likelihood evaluations in the Newton passes / whole step time (a lower bound on "
                    "the pass rate: the step also ranks, tabulates, scans the variance and combines); "
                    "the FP64 path starts its FP64 passes from the root of an FP32 search, counted apart",
            "f32c_search_phase_pairs_per_s": search_rate,
            "search_phase_note": "pair-likelihood evaluations / mean in-kernel Newton-phase time per subset "
                                 "(in-kernel timer stamps; all K subsets run concurrently, one per SM)"},
        "phases_f32c": phase_summary(ph),
        "fp64": {"value": val64, "unit": "pairs/s", "ms_per_step": 1e3 * t64 / steps64, "steps": steps64,
                 "kernel_ms": kms64_mean},
        "f32c_over_f64": value / val64,
        "e2e": {"value": world * n * e2e_steps / te if world == 1 else None, "unit": "pairs/s",
                "h2d_bytes_per_step": 2 * n * d.u.itemsize, "d2h_bytes_per_step": d.K * (8 + 8 + 4) + 8,
                "call": "copula_fit_host (pinned host u, v in, read by the fit kernel over the host link; "
                        "theta, var, status, combined out)"},
        "gpu_launches": launches * args.steps,
        "kernel_ms_f32c": kms32_mean,
        "roofline": roof,
    }
    if world > 1:
        line["e2e"]["value"] = world * n * e2e_steps / te
    if clk is not None:
        line["clocks"] = clk
    if not args.no_serving and world == 1:
        line["serving"] = serving_bench()
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(d)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# serving: Poisson arrivals of fit requests (family uniform over the three,
# Kendall tau ~ U[0.1, 0.8], n log-uniform in [1e4, 1e7] FP32 pairs, K = n/1e4)
# against the continuous-batching server under a 64 GB HBM budget
# ---------------------------------------------------------------------------

def serving_bench(pool_size=48, rates=(500, 1000, 2000, 4000, 8000), seconds=3.0, seed=1605535, solo_rounds=3):
    import threading

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
    # warm-up and unloaded latency: one request at a time
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


def run_mixed(args):
    """4096 datasets (family uniform, tau U[0.1,0.8], n log-uniform [1e3,1e6],
    K = max(1, n/1e4)) fitted by one CUDA-graph replay per step."""
    import torch

    import paper_1609_05530_gb300 as cg
    from copula_synth import device as dsyn

    bt = dsyn.mixed_batch(B=4096)
    n = int(bt["dataset_offsets"][-1])
    out = {}
    for prec in ("f32c", "f64"):
        plan = cg.BatchPlan(bt["families"], bt["dataset_offsets"], bt["subset_offsets"], bt["dataset_subset_start"],
                            precision=prec)
        gr = plan.capture(bt["u"], bt["v"])
        steps = args.steps if prec == "f32c" else max(3, args.steps // 10)
        for _ in range(args.warmup):
            gr.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            gr.replay()
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        out[prec] = {"value": n * steps / t, "ms_per_step": 1e3 * t / steps, "steps": steps}
        plan.close()
    line = {"metric": METRIC, "value": out["f32c"]["value"], "unit": "pairs/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": out["f32c"]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "mixed_4096_datasets", "n": n, "datasets": 4096,
                       "subsets": int(bt["dataset_subset_start"][-1]),
                       "step": "one CUDA-graph replay of the batched fit", "l2": "inputs (4.7 GB) larger than L2"},
            "fp64": out["f64"], "f32c_over_f64": out["f32c"]["value"] / out["f64"]["value"]}
    print(json.dumps(line), flush=True)
    return 0


def phase_summary(ph):
    """Mean per-subset time in each phase (us) from the in-kernel stamps."""
    if ph is None or ph.size == 0:
        return None
    dt = np.diff(ph, axis=1) / 1e3
    return {"ranks_us": float(dt[:, 0].mean()), "search_us": float(dt[:, 1].mean()),
            "variance_us": float(dt[:, 2].mean()), "subset_total_us": float((ph[:, 3] - ph[:, 0]).mean() / 1e3),
            "kernel_span_us": float((ph[:, 3].max() - ph[:, 0].min()) / 1e3)}


# Algorithmic 32-bit lane operations per unit of the fused fit kernel: per
# key per 4-bit radix pass (histogram walk + scatter walk),
# per pair per Frank likelihood pass (density terms + two compensated sums),
# per rank per pass (exp-table entry), per pair for pi, and per pair for the
# sandwich variance (two evaluations with mixed partials, two suffix scans,
# two sums).  MUFU operations per pair-pass / per rank-pass / per pair of
# variance, for the transcendental-rate figure.
OPS_KEY_PASS = 16.0
OPS_PAIR_PASS = 40.0
OPS_RANK_PASS = 8.0
OPS_PI = 4.0
OPS_VAR = 140.0
MUFU_PAIR_PASS, MUFU_RANK_PASS, MUFU_VAR = 1.0, 1.0, 3.0


def varying_digits(x, off):
    """4-bit digits of the order-preserving keys not constant within each subset."""
    if x.dtype == np.float64:
        b = x.view(np.uint64)
        top = np.uint64(1) << np.uint64(63)
        key = np.where(b & top, ~b, b | top)
        nd = 16
    else:
        b = x.view(np.uint32)
        key = np.where(b & 0x80000000, ~b, b | 0x80000000).astype(np.uint32)
        nd = 8
    out = []
    for k in range(len(off) - 1):
        s = key[off[k]:off[k + 1]]
        diff = np.bitwise_or.reduce(s ^ s[0])
        out.append(sum(1 for j in range(nd) if (int(diff) >> (4 * j)) & 15))
    return np.array(out, dtype=np.float64)


def roofline(d, diag, kernel_ms, clk, peaks, peak_kind):
    """Roofline of the fused per-subset kernel (the only large kernel of a step).

    The data are read from HBM once (8 B/pair) and every later pass runs out of
    shared memory, so the binding unit is the SM's 32-bit issue slots; the
    algorithmic work is counted in lane operations per the constants above,
    against 152 SMs x 128 lanes x the SM clock seen under load.  The HBM and
    MUFU fractions (bytes at HBM peak, transcendentals at the MUFU rate) are
    reported beside it."""
    m = np.diff(d.offsets).astype(np.float64)
    it = diag.iters.cpu().numpy().astype(np.float64)
    digits = varying_digits(d.u, d.offsets) + varying_digits(d.v, d.offsets)
    ops = float((m * digits * OPS_KEY_PASS + m * (OPS_PI + OPS_VAR) + m * it * (OPS_PAIR_PASS + OPS_RANK_PASS)).sum())
    mufu = float((m * it * (MUFU_PAIR_PASS + MUFU_RANK_PASS) + m * MUFU_VAR).sum())
    sm_mhz = (clk or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    peak = 152 * 128 * sm_mhz * 1e6 / 1e12  # T lane-ops/s
    secs = kernel_ms * 1e-3
    achieved = ops / secs / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
            "traffic": captured_traffic("resident") if d.name == "frank_theta5_n1e6_K100" else None,
            "traffic_unit": "bytes/launch", "kernel": "resident_kernel<float," + ("uint64_t" if d.u.dtype == np.float64 else "uint32_t") + ",512>",
            "peak_basis": f"152 SMs x 128 32-bit lanes x {sm_mhz:.0f} MHz median SM clock under load (derived)",
            "work_per_launch": {"lane_ops": ops, "mufu_ops": mufu, "hbm_bytes": 8.0 * d.n},
            "hbm_frac": (8.0 * d.n / secs / 1e9) / peaks.get("hbm_gbs", 6800.0), "hbm_peak_kind": peak_kind,
            "mufu_frac": mufu / secs / (152 * 16 * sm_mhz * 1e6)}


def run_gumbel(args):
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
    clocks = ClockSampler(0, enabled=not args.no_clocks)
    clocks.start()
    for prec in ("f32c", "f64"):
        o = cg.make_opts(prec)
        steps = args.steps if prec == "f32c" else max(3, args.steps // 5)
        for _ in range(args.warmup):
            cg.fit(u, v, off, cg.GUMBEL, ctx=ctx, opts=o)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(steps):
            r = cg.fit(u, v, off, cg.GUMBEL, ctx=ctx, opts=o)
        ev[1].record()
        torch.cuda.synchronize()
        t = ev[0].elapsed_time(ev[1]) / 1e3
        launches = ctx.launches()
        # stage spans (events inside the library, on the launching stream)
        ctx.set_timing(True)
        spans, total = [], []
        for _ in range(max(3, steps // 2)):
            cg.fit(u, v, off, cg.GUMBEL, ctx=ctx, opts=o)
            total.append(ctx.kernel_ms())
            spans.append(ctx.stage_ms())
        ctx.set_timing(False)
        _, diag = cg.fit_ex(u, v, off, cg.GUMBEL, ctx=ctx, opts=o)
        it = diag.iters.cpu().numpy().astype(np.float64)
        big = m > cg.MAX_SUBSET
        sp = np.mean(np.array(spans), axis=0)
        out[prec] = {"value": n * steps / t, "ms_per_step": 1e3 * t / steps, "steps": steps,
                     "launches_per_step": launches, "kernel_span_ms": float(np.mean(total)),
                     "stages_ms": {"shared_memory_subsets_and_setup": float(np.mean(total) - sp.sum()),
                                   "ranks_u": float(sp[0]), "ranks_v": float(sp[1]), "pi": float(sp[2]),
                                   "fit_kernel": float(sp[3])},
                     "newton_passes_per_pair_stream": float((m[big] * it[big]).sum() / m[big].sum()),
                     "theta_combined": float(r.combined.item())}
    clk = clocks.stop()
    peaks, peak_kind = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    f = out["f32c"]
    st = f["stages_ms"]
    nb = float(m[m > cg.MAX_SUBSET].sum())
    # algorithmic HBM bytes per launch sequence: a column rank reads the value
    # and writes the rank (8 B/pair); the fit kernel reads pi and the table
    # once per Newton pass and twice for the variance, and writes the table
    # (8 B/pair per pass + 4 B)
    algo = {"ranks_u": 8.0 * nb, "ranks_v": 8.0 * nb,
            "fit_kernel": nb * (4.0 + 8.0 * (f["newton_passes_per_pair_stream"] + 2.0))}
    dom = max(algo, key=lambda k: st[k])
    achieved = algo[dom] / (st[dom] * 1e-3) / 1e9
    # e2e: host buffers through copula_fit_host (800 MB in per step)
    hu, hv = u.cpu().pin_memory(), v.cpu().pin_memory()
    outs = (np.empty(K), np.empty(K), np.empty(K, dtype=np.int32), np.empty(1))
    cg.fit_host(hu, hv, off, cg.GUMBEL, ctx=ctx, opts=cg.make_opts("f32c"), out=outs)
    e2e_steps = max(3, args.steps // 5)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        cg.fit_host(hu, hv, off, cg.GUMBEL, ctx=ctx, opts=cg.make_opts("f32c"), out=outs)
    te = time.perf_counter() - t0
    line = {"metric": METRIC, "value": f["value"], "unit": "pairs/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": f["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "gumbel_theta2_n1e8_K1000_lognormal" if args.scale == 1.0
                       else f"gumbel_theta2_n{n}_K{K}_lognormal", "n": n, "K": K,
                       "streaming_subsets": int((m > cg.MAX_SUBSET).sum()), "largest_subset": int(m.max()),
                       "l2": "inputs (800 MB) larger than L2"},
            "f32c": f, "fp64": out["f64"], "f32c_over_f64": f["value"] / out["f64"]["value"],
            "e2e": {"value": n * e2e_steps / te, "unit": "pairs/s", "h2d_bytes_per_step": 8 * n,
                    "d2h_bytes_per_step": K * 20 + 8, "call": "copula_fit_host"},
            "gpu_launches": f["launches_per_step"] * args.steps,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm,
                         "traffic": captured_traffic("stream") if dom == "fit_kernel" and args.scale == 1.0 else None,
                         "traffic_unit": "bytes/launch", "peak_kind": peak_kind,
                         "algorithmic_bytes": algo[dom]}}
    if clk is not None:
        line["clocks"] = clk
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "mixed_4096":
        return run_mixed(args)
    if args.workload == "gumbel_1e8":
        return run_gumbel(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
