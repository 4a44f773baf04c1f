"""Seeded synthetic inputs drawn directly on the GPU (for workloads too large
to draw on the host in reasonable time).

Same samplers as the host module -- correlated normals through Phi for the
Gaussian copula, conditional inversion for Frank, Marshall-Olkin with a
positive-stable frailty for Gumbel -- computed in FP64 with torch's
Philox4x32-10 CUDA generator and stored as FP32.  Holds none of the
estimator's arithmetic.  The host oracle checks these workloads on copies of
sampled datasets.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import FRANK, GAUSSIAN, GUMBEL, equal_offsets, theta_of_tau


def sample(family: int, theta: float, n: int, g: torch.Generator, device="cuda"):
    """n pairs (u, v) in FP64 on the device, drawn from C(.;theta)."""
    kw = dict(generator=g, device=device, dtype=torch.float64)
    if family == GAUSSIAN:
        z1 = torch.randn(n, **kw)
        z2 = torch.randn(n, **kw)
        y = theta * z1 + math.sqrt(1.0 - theta * theta) * z2
        return torch.special.ndtr(z1), torch.special.ndtr(y)
    if family == FRANK:
        u = torch.rand(n, **kw)
        p = torch.rand(n, **kw)
        if theta == 0.0:
            return u, p
        v = -torch.log1p(p * math.expm1(-theta) / (p + (1.0 - p) * torch.exp(-theta * u))) / theta
        return u, v
    if family == GUMBEL:
        alpha = 1.0 / theta
        th = torch.rand(n, **kw) * math.pi
        w = -torch.log(torch.rand(n, **kw))
        if alpha == 1.0:
            V = torch.ones(n, **{k: kw[k] for k in ("device", "dtype")})
        else:
            V = (torch.sin(alpha * th) / torch.sin(th) ** (1.0 / alpha)) * \
                (torch.sin((1.0 - alpha) * th) / w) ** ((1.0 - alpha) / alpha)
        e1 = -torch.log(torch.rand(n, **kw))
        e2 = -torch.log(torch.rand(n, **kw))
        return torch.exp(-(e1 / V) ** alpha), torch.exp(-(e2 / V) ** alpha)
    raise ValueError(family)


def mixed_batch(B: int = 4096, seed: int = 1605534, n_lo: float = 1e3, n_hi: float = 1e6,
                m_target: float = 1e4, device="cuda"):
    """B datasets: family uniform over the three, Kendall tau ~ U[0.1, 0.8]
    mapped to theta, n log-uniform in [n_lo, n_hi], K = max(1, floor(n/m_target))
    equal subsets; concatenated FP32 columns on the device.

    Returns dict(u, v, families, thetas, dataset_offsets, subset_offsets,
    dataset_subset_start) (offsets as host int64 arrays)."""
    rng = np.random.Generator(np.random.Philox(seed))
    fams = rng.integers(0, 3, B)
    taus = rng.uniform(0.1, 0.8, B)
    ns = np.floor(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), B))).astype(np.int64)
    thetas = np.array([theta_of_tau(int(f), float(t)) for f, t in zip(fams, taus)])
    dofs = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
    n = int(dofs[-1])
    u = torch.empty(n, dtype=torch.float32, device=device)
    v = torch.empty(n, dtype=torch.float32, device=device)
    sub = [np.array([0], dtype=np.int64)]
    starts = [0]
    g = torch.Generator(device=device)
    for b in range(B):
        g.manual_seed(seed * 7919 + b + 1)
        ub, vb = sample(int(fams[b]), float(thetas[b]), int(ns[b]), g, device)
        u[dofs[b]:dofs[b + 1]] = ub.to(torch.float32)
        v[dofs[b]:dofs[b + 1]] = vb.to(torch.float32)
        K = max(1, int(ns[b] // m_target))
        sub.append(equal_offsets(int(ns[b]), K)[1:] + dofs[b])
        starts.append(starts[-1] + K)
    return dict(u=u, v=v, families=fams.astype(np.int32), thetas=thetas, dataset_offsets=dofs,
                subset_offsets=np.concatenate(sub).astype(np.int64),
                dataset_subset_start=np.array(starts, dtype=np.int64))


def equal_batch(family: int, theta: float, m: int, S: int, seed: int, device="cuda"):
    """S subsets of m pairs from one copula as one dataset (for tuning)."""
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    u, v = sample(family, theta, m * S, g, device)
    return u.to(torch.float32), v.to(torch.float32), equal_offsets(m * S, S)


def gumbel_lognormal(n: int = 100_000_000, K: int = 1000, sigma: float = 1.0, seed: int = 1605533,
                     chunk: int = 1 << 24, device="cuda"):
    """Gumbel theta = 2, n FP32 pairs drawn on the device in chunks of 2^24
    (one seeded generator per chunk), split into K subsets of lognormal(sigma)
    relative size (the same offsets as the host workload of this name).

    Returns (u, v, subset_offsets) with the offsets as a host int64 array."""
    from . import lognormal_offsets, rng
    off = lognormal_offsets(n, K, sigma, rng(seed + 100))
    u = torch.empty(n, dtype=torch.float32, device=device)
    v = torch.empty(n, dtype=torch.float32, device=device)
    g = torch.Generator(device=device)
    for i, s in enumerate(range(0, n, chunk)):
        g.manual_seed(seed * 7919 + i + 1)
        c = min(chunk, n - s)
        a, b = sample(GUMBEL, 2.0, c, g, device)
        u[s:s + c] = a.to(torch.float32)
        v[s:s + c] = b.to(torch.float32)
        del a, b
    return u, v, off
