"""Autotuner for the fused per-subset fit.

A subset of m rows runs in one CTA of 128, 256 or 512 threads (hence
ceil(m / threads) points per thread); smaller CTAs let two or more subsets
share an SM where their shared memory and registers allow (256 threads: two
per SM up to about 10,500 rows), which hides each CTA's serial steps (the
thread-0 Newton updates, the block reductions) behind the other's work.
Subsets of different block sizes run in separate launches, one after
another, so what matters is the whole batch, not each size alone: the tuner
therefore times whole candidate tables -- the built-in rule (128 threads up
to 1,536 rows, 256 up to 6,144, 512 above) and tables that move the
256-thread bound to each of a ladder of sizes, with and without the
128-thread bucket -- as CUDA-graph replays of a mixed-size batch of the
family (n log-uniform in [1e3, 1e6], K = max(1, n / 1e4), the shape of the
batched workloads), and keeps the fastest.  The families are tuned apart
because their per-pass costs differ (the Gaussian has none: its Newton
iteration runs on two sums).  The tables -- (largest m, threads) per bucket
and family -- are installed with copula_ctx_set_family_blocks and cached per
GPU model, precision, storage type and family in a JSON file next to the
built library ([] is the built-in rule).  The subset-to-CTA schedule itself
(longest subset first through an atomic job counter) needs no tuning.
"""
from __future__ import annotations

import json
import os
import statistics

import numpy as np

from . import FRANK, GAUSSIAN, GUMBEL, Context, context, set_blocks
from .build import OUT_DIR

FAMILY_CASES = ((GAUSSIAN, 0.5), (FRANK, 5.0), (GUMBEL, 2.0))
BOUNDS_256 = (6144, 8192, 9216, 9728, 10240, 10496, 11264, 12288, 16384, 20480)
CACHE = os.path.join(OUT_DIR, "autotune.json")


def candidates():
    """Candidate tables: the built-in rule ([]) and, for each bound T of the
    ladder, 256 threads up to T (with and without 128 up to 1,536) and 512
    above."""
    out = [[]]
    for t in BOUNDS_256:
        hi = [(20480, 512)] if t < 20480 else []
        out.append([(1536, 128), (t, 256)] + hi)
        out.append([(t, 256)] + hi)
    return out


def _key(precision: str, dtype: str, family: int) -> str:
    import torch
    return f"{torch.cuda.get_device_name()}|{precision}|{dtype}|family{int(family)}"


def mixed_family_batch(family: int, theta: float, dtype: str = "f32", B: int = 256, seed: int = 4242):
    """B datasets of one family: n log-uniform in [1e3, 1e6], K = max(1, n /
    1e4) equal subsets, drawn on the device."""
    import torch

    from copula_synth import equal_offsets
    from copula_synth import device as dev
    rng = np.random.Generator(np.random.Philox(seed + family))
    ns = np.floor(np.exp(rng.uniform(np.log(1e3), np.log(1e6), B))).astype(np.int64)
    dofs = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
    sub, starts = [np.array([0], dtype=np.int64)], [0]
    for b in range(B):
        K = max(1, int(ns[b] // 10_000))
        sub.append(equal_offsets(int(ns[b]), K)[1:] + dofs[b])
        starts.append(starts[-1] + K)
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    u, v = dev.sample(family, theta, int(dofs[-1]), g)
    u, v = (u.double(), v.double()) if dtype == "f64" else (u.float(), v.float())
    return u, v, dofs, np.concatenate(sub).astype(np.int64), np.array(starts, dtype=np.int64)


def batch_ms(u, v, dofs, soff, dss, families, precision, table, family, reps=5):
    """Median CUDA-graph replay time (ms) of a batched fit with `table`
    installed for `family` on a fresh context ([] = the built-in rule)."""
    import torch

    from . import BatchPlan
    ctx = Context()
    if table:
        set_blocks(table, ctx, family=family)
    plan = BatchPlan(families, dofs, soff, dss, precision=precision, ctx=ctx)
    g = plan.capture(u, v)
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    del g
    plan.close()
    ctx.close()
    return statistics.median(ts)


def tune_family(family: int, theta: float, precision: str = "f32c", dtype: str = "f32", reps: int = 5):
    """(table, timings): the fastest candidate table on the family's mixed-size
    batch ([] if the built-in rule is) and every candidate's time."""
    import torch
    u, v, dofs, soff, dss = mixed_family_batch(family, theta, dtype)
    fams = [family] * (len(dofs) - 1)
    timings = []
    for table in candidates():
        timings.append((table, batch_ms(u, v, dofs, soff, dss, fams, precision, table, family, reps)))
    del u, v
    torch.cuda.empty_cache()
    best = min(timings, key=lambda x: x[1])
    return best[0], [{"table": t, "ms": ms} for t, ms in timings]


def tune(precision: str = "f32c", dtype: str = "f32", reps: int = 5):
    """Tables of every family: {family: (table, timings)}."""
    return {fam: tune_family(fam, th, precision, dtype, reps) for fam, th in FAMILY_CASES}


def load_or_tune(precision: str = "f32c", dtype: str = "f32", ctx: Context | None = None, retune: bool = False):
    """Installs the cached tables for this GPU (tuning first where absent);
    returns {family: table}."""
    ctx = ctx or context()
    cache = {}
    if os.path.exists(CACHE):
        with open(CACHE) as f:
            cache = json.load(f)
    out = {}
    dirty = False
    for fam, th in FAMILY_CASES:
        key = _key(precision, dtype, fam)
        if retune or key not in cache:
            table, timings = tune_family(fam, th, precision, dtype)
            cache[key] = {"table": table, "timings_ms": timings}
            dirty = True
        out[fam] = [tuple(x) for x in cache[key]["table"]]
        set_blocks(out[fam], ctx, family=fam)
    if dirty:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1)
    return out
