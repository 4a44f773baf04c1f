"""Autotuner for the fused per-subset fit.

For each subset-size bucket it times the fit kernel with 128, 256 and 512
threads per subset (hence ceil(m / threads) points per thread) on batches of
synthetic Frank and Gumbel subsets large enough to fill the GPU, and keeps the
fastest.  The resulting table -- (largest m, threads) per bucket -- is
installed with copula_ctx_set_blocks and cached per GPU model, precision and
storage type in a JSON file next to the built library.  The subset-to-CTA
schedule itself (longest subset first through an atomic job counter) needs
no tuning.
"""
from __future__ import annotations

import json
import os
import statistics

import numpy as np

from . import FRANK, GUMBEL, Context, context, fit, make_opts, set_blocks
from .build import OUT_DIR

CANDIDATES = (128, 256, 512)
SIZES = (384, 1024, 2048, 4096, 8192, 14336, 20480)
CACHE = os.path.join(OUT_DIR, "autotune.json")


def _key(precision: str, dtype: str) -> str:
    import torch
    return f"{torch.cuda.get_device_name()}|{precision}|{dtype}"


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


def tune(precision: str = "f32c", dtype: str = "f32", reps: int = 5, ctx: Context | None = None, sms: int = 152):
    """Returns (table, timings): table = [(largest m, threads), ...]."""
    import torch

    from copula_synth import device as dev

    ctx = ctx or context()
    best, timings = [], {}
    for i, m in enumerate(SIZES):
        S = 2 * sms  # two subsets per SM
        t = {}
        for fam, theta in ((FRANK, 5.0), (GUMBEL, 2.0)):
            u, v, off = dev.equal_batch(fam, theta, m, S, seed=1000 + i)
            if dtype == "f64":
                u, v = u.double(), v.double()
            for b in CANDIDATES:
                t[b] = t.get(b, 0.0) + _time_block(u, v, off, fam, precision, b, ctx, reps)
            del u, v
        torch.cuda.empty_cache()
        timings[m] = t
        best.append(min(t, key=t.get))
    # bucket bounds half-way (geometrically) between the tuned sizes
    table = []
    for i, m in enumerate(SIZES):
        hi = SIZES[-1] if i + 1 == len(SIZES) else int(np.sqrt(m * SIZES[i + 1]))
        if table and table[-1][1] == best[i]:
            table[-1] = (hi, best[i])
        else:
            table.append((hi, best[i]))
    return table, timings


def load_or_tune(precision: str = "f32c", dtype: str = "f32", ctx: Context | None = None, retune: bool = False):
    """Installs the cached table for this GPU (tuning first if absent)."""
    ctx = ctx or context()
    cache = {}
    if os.path.exists(CACHE):
        with open(CACHE) as f:
            cache = json.load(f)
    key = _key(precision, dtype)
    if retune or key not in cache:
        table, timings = tune(precision, dtype, ctx=ctx)
        cache[key] = {"table": table, "timings_ms": {str(k): v for k, v in timings.items()}}
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1)
    table = [tuple(x) for x in cache[key]["table"]]
    set_blocks(table, ctx)
    return table
