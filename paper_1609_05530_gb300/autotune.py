"""Autotuner for the fused per-subset fit.

For each family and subset-size bucket it times the fit kernel with 128, 256
and 512 threads per subset (hence ceil(m / threads) points per thread, and
one or two subsets per SM where shared memory and registers allow) on
batches of synthetic subsets of that family, eight per SM, so that the
measurement is of throughput and not of the batch's tail, and keeps the
fastest.  The families are tuned apart because their per-pass costs differ
(the Gaussian has none: its Newton iteration runs on two sums).  Subsets of
different block sizes run in separate launches, one after another, so a
table that is faster size by size can still lose on a batch of mixed sizes:
each family's table is therefore checked on a mixed-size batch of that family
against the built-in rule and replaced by the built-in rule (an empty table)
if it is not faster.  The resulting tables -- (largest m, threads) per bucket
and family -- are installed with copula_ctx_set_family_blocks and cached per
GPU model, precision, storage type and family in a JSON file next to the
built library.  The subset-to-CTA schedule itself (longest subset first
through an atomic job counter) needs no tuning.
"""
from __future__ import annotations

import json
import os
import statistics

import numpy as np

from . import FRANK, GAUSSIAN, GUMBEL, Context, context, fit, make_opts, set_blocks
from .build import OUT_DIR

CANDIDATES = (128, 256, 512)
SIZES = (384, 1024, 2048, 4096, 8192, 10240, 14336, 20480)
FAMILY_CASES = ((GAUSSIAN, 0.5), (FRANK, 5.0), (GUMBEL, 2.0))
CACHE = os.path.join(OUT_DIR, "autotune.json")


def _key(precision: str, dtype: str, family: int) -> str:
    import torch
    return f"{torch.cuda.get_device_name()}|{precision}|{dtype}|family{int(family)}"


def _time_block(u, v, off, family, precision, block, ctx, reps):
    opts = make_opts(precision, block=block)
    for _ in range(2):
        fit(u, v, off, family, ctx=ctx, opts=opts)
    ctx.set_timing(True)
    ts = []
    for _ in range(reps):
        fit(u, v, off, family, ctx=ctx, opts=opts)
        ts.append(ctx.kernel_ms())
    ctx.set_timing(False)
    return statistics.median(ts)


def _table(best):
    """Bucket bounds half-way (geometrically) between the tuned sizes."""
    table = []
    for i, m in enumerate(SIZES):
        hi = SIZES[-1] if i + 1 == len(SIZES) else int(np.sqrt(m * SIZES[i + 1]))
        if table and table[-1][1] == best[i]:
            table[-1] = (hi, best[i])
        else:
            table.append((hi, best[i]))
    return table


def tune_family(family: int, theta: float, precision: str = "f32c", dtype: str = "f32", reps: int = 5,
                ctx: Context | None = None, sms: int = 152):
    """Returns (table, timings) for one family: table = [(largest m, threads), ...]."""
    import torch

    from copula_synth import device as dev

    ctx = ctx or context()
    best, timings = [], {}
    for i, m in enumerate(SIZES):
        S = 8 * sms  # eight subsets per SM: throughput, not the tail
        u, v, off = dev.equal_batch(family, theta, m, S, seed=1000 + 10 * i + family)
        if dtype == "f64":
            u, v = u.double(), v.double()
        t = {b: _time_block(u, v, off, family, precision, b, ctx, reps) for b in CANDIDATES}
        del u, v
        torch.cuda.empty_cache()
        timings[m] = t
        best.append(min(t, key=t.get))
    return _table(best), timings


def _batch_ms(u, v, dofs, soff, dss, families, precision, table, family, reps):
    """Median CUDA-graph replay time of a batched fit with `table` installed
    for `family` on a fresh context ([] = the built-in rule)."""
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


def validate_family(family: int, theta: float, table, precision: str = "f32c", dtype: str = "f32", reps: int = 5,
                    B: int = 256, seed: int = 4242):
    """(table or [], timings): the tuned table if it fits a mixed-size batch
    of the family (n log-uniform in [1e3, 1e6], K = max(1, n / 1e4), as the
    batched workloads) faster than the built-in rule, else [] (the rule)."""
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
    soff = np.concatenate(sub).astype(np.int64)
    dss = np.array(starts, dtype=np.int64)
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    u, v = dev.sample(family, theta, int(dofs[-1]), g)
    u, v = (u.double(), v.double()) if dtype == "f64" else (u.float(), v.float())
    fams = [family] * B
    t_rule = _batch_ms(u, v, dofs, soff, dss, fams, precision, [], family, reps)
    t_tuned = _batch_ms(u, v, dofs, soff, dss, fams, precision, table, family, reps) if table else t_rule
    del u, v
    torch.cuda.empty_cache()
    return (table if t_tuned < t_rule else []), {"rule_ms": t_rule, "tuned_ms": t_tuned}


def tune(precision: str = "f32c", dtype: str = "f32", reps: int = 5, ctx: Context | None = None, sms: int = 152):
    """Tables of every family: {family: (table, timings)}; a table that loses
    to the built-in rule on a mixed-size batch of its family is [] (the rule)."""
    out = {}
    for fam, th in FAMILY_CASES:
        table, timings = tune_family(fam, th, precision, dtype, reps, ctx, sms)
        table, check = validate_family(fam, th, table, precision, dtype)
        timings["mixed_batch_check"] = check
        out[fam] = (table, timings)
    return out


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
            table, timings = tune_family(fam, th, precision, dtype, ctx=ctx)
            table, check = validate_family(fam, th, table, precision, dtype)
            timings["mixed_batch_check"] = check
            cache[key] = {"table": table, "timings_ms": {str(k): v for k, v in timings.items()}}
            dirty = True
        out[fam] = [tuple(x) for x in cache[key]["table"]]
        set_blocks(out[fam], ctx, family=fam)
    if dirty:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1)
    return out
