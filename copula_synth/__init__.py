"""Seeded synthetic inputs for the copula estimator (shared by tests and bench).

This module only draws data; it holds none of the estimator's arithmetic
(no ranks, no likelihood, no optimiser, no combine).  Both the CPU oracle and
the CUDA path are fed from it, so that they see identical inputs.

Random numbers come from numpy's Philox4x32-10 counter-based generator
(Salmon et al., SC'11), seeded per workload.  Pairs are drawn in FP64 from the
copula itself, as in the paper's simulation design (Section 2.5), then stored
in the requested dtype:

* Gaussian (Eq. 7-8): correlated standard normals mapped through Phi.
* Frank (Eq. 10): conditional inversion, v = C_{2|1}^{-1}(p | u).
* Gumbel (Eq. 11): Marshall-Olkin with a positive-stable frailty
  V ~ S(alpha = 1/theta) drawn by the Chambers-Mallows-Stuck / Kanter form,
  then U_i = exp(-(E_i / V)^alpha).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy import integrate, optimize, special

GAUSSIAN, FRANK, GUMBEL = 0, 1, 2
FAMILY_NAMES = {GAUSSIAN: "gaussian", FRANK: "frank", GUMBEL: "gumbel"}
BASE_SEED = 1605530


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


# ----------------------------------------------------------------------------
# Kendall's tau <-> parameter maps (textbook closed forms; used to pick the
# generating parameter of a workload from its tau).
# ----------------------------------------------------------------------------

def _debye1(t: float) -> float:
    if t == 0.0:
        return 1.0
    val, _ = integrate.quad(lambda s: s / math.expm1(s) if s != 0 else 1.0, 0.0, abs(t),
                            epsabs=1e-14, epsrel=1e-13)
    d = val / abs(t)
    return d if t > 0 else d + abs(t) / 2.0


def tau_of(family: int, theta: float) -> float:
    if family == GAUSSIAN:
        return 2.0 / math.pi * math.asin(theta)
    if family == GUMBEL:
        return 1.0 - 1.0 / theta
    if theta == 0.0:
        return 0.0
    return 1.0 - 4.0 / theta + 4.0 * _debye1(theta) / theta


def theta_of_tau(family: int, tau: float) -> float:
    if family == GAUSSIAN:
        return math.sin(math.pi * tau / 2.0)
    if family == GUMBEL:
        return 1.0 / (1.0 - tau)
    if tau == 0.0:
        return 0.0
    lo, hi = (1e-9, 200.0) if tau > 0 else (-200.0, -1e-9)
    return optimize.brentq(lambda t: tau_of(FRANK, t) - tau, lo, hi, xtol=1e-13, rtol=1e-14)


# ----------------------------------------------------------------------------
# Samplers (FP64).
# ----------------------------------------------------------------------------

def sample(family: int, theta: float, n: int, g: np.random.Generator):
    """n pairs (u, v) in FP64 drawn from the copula C(.;theta)."""
    if family == GAUSSIAN:
        z1 = g.standard_normal(n)
        z2 = g.standard_normal(n)
        x = z1
        y = theta * z1 + math.sqrt(1.0 - theta * theta) * z2
        return special.ndtr(x), special.ndtr(y)
    if family == FRANK:
        u = g.random(n)
        p = g.random(n)
        if theta == 0.0:
            return u, p
        # conditional inversion of C_{2|1}(v|u) = p
        v = -np.log1p(p * np.expm1(-theta) / (p + (1.0 - p) * np.exp(-theta * u))) / theta
        return u, v
    if family == GUMBEL:
        alpha = 1.0 / theta
        th = g.random(n) * math.pi
        w = g.exponential(1.0, n)
        if alpha == 1.0:
            V = np.ones(n)
        else:
            V = (np.sin(alpha * th) / np.sin(th) ** (1.0 / alpha)) * \
                (np.sin((1.0 - alpha) * th) / w) ** ((1.0 - alpha) / alpha)
        e1 = g.exponential(1.0, n)
        e2 = g.exponential(1.0, n)
        return np.exp(-(e1 / V) ** alpha), np.exp(-(e2 / V) ** alpha)
    raise ValueError(family)


# ----------------------------------------------------------------------------
# Partitions (Eq. 14: contiguous row blocks).
# ----------------------------------------------------------------------------

def equal_offsets(n: int, K: int) -> np.ndarray:
    """K contiguous blocks; the first n mod K blocks get one extra row."""
    base, extra = divmod(n, K)
    sizes = np.full(K, base, dtype=np.int64)
    sizes[:extra] += 1
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def lognormal_offsets(n: int, K: int, sigma: float, g: np.random.Generator, min_m: int = 2):
    """K blocks with lognormal(sigma) relative sizes, rounded by largest remainder
    to sum exactly to n, each at least min_m."""
    w = np.exp(sigma * g.standard_normal(K))
    avail = n - min_m * K
    raw = w / w.sum() * avail
    fl = np.floor(raw).astype(np.int64)
    rem = avail - int(fl.sum())
    order = np.argsort(-(raw - fl), kind="stable")
    fl[order[:rem]] += 1
    sizes = fl + min_m
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


# ----------------------------------------------------------------------------
# Workloads.
# ----------------------------------------------------------------------------

@dataclass
class Dataset:
    family: int
    theta: float
    u: np.ndarray
    v: np.ndarray
    offsets: np.ndarray          # K+1 int64 row offsets (Eq. 14)
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.u.shape[0])

    @property
    def K(self) -> int:
        return int(self.offsets.shape[0] - 1)


def make_dataset(family: int, theta: float, n: int, K: int, dtype=np.float32, seed: int = BASE_SEED,
                 offsets=None, name: str = "") -> Dataset:
    g = rng(seed)
    u, v = sample(family, theta, n, g)
    off = equal_offsets(n, K) if offsets is None else np.asarray(offsets, dtype=np.int64)
    return Dataset(family, theta, u.astype(dtype), v.astype(dtype), off, name)


def gaussian_10k(dtype=np.float64, K: int = 10) -> Dataset:
    """Gaussian rho=0.5, n=10,000 pairs in FP64, K equal subsets."""
    return make_dataset(GAUSSIAN, 0.5, 10_000, K, dtype, BASE_SEED + 1, name="gaussian_rho0.5_n1e4")


def frank_1m(dtype=np.float32) -> Dataset:
    """Frank theta=5, n=1,000,000 pairs stored FP32, K=100 equal subsets."""
    return make_dataset(FRANK, 5.0, 1_000_000, 100, dtype, BASE_SEED + 2, name="frank_theta5_n1e6_K100")


def gumbel_lognormal(n: int = 100_000_000, K: int = 1000, sigma: float = 1.0, dtype=np.float32,
                     seed: int = BASE_SEED + 3) -> Dataset:
    """Gumbel theta=2, n pairs stored FP32, K lognormal(sigma)-sized subsets."""
    g = rng(seed)
    off = lognormal_offsets(n, K, sigma, rng(seed + 100))
    u, v = sample(GUMBEL, 2.0, n, g)
    return Dataset(GUMBEL, 2.0, u.astype(dtype), v.astype(dtype), off,
                   f"gumbel_theta2_n{n}_K{K}_lognormal")


def mixed_batch(B: int = 4096, n_lo: float = 1e3, n_hi: float = 1e6, seed: int = BASE_SEED + 4,
                dtype=np.float32, m_target: float = 1e4):
    """B independent datasets: family uniform over the three, tau ~ U[0.1, 0.8],
    n log-uniform in [n_lo, n_hi], K = max(1, floor(n / m_target))."""
    g = rng(seed)
    fams = g.integers(0, 3, B)
    taus = g.uniform(0.1, 0.8, B)
    ns = np.floor(np.exp(g.uniform(math.log(n_lo), math.log(n_hi), B))).astype(np.int64)
    out = []
    for b in range(B):
        fam = int(fams[b])
        th = theta_of_tau(fam, float(taus[b]))
        n = int(ns[b])
        K = max(1, int(n // m_target))
        out.append(make_dataset(fam, th, n, K, dtype, seed * 7919 + b + 1,
                                name=f"mix{b}_{FAMILY_NAMES[fam]}"))
    return out


def pack_batch(datasets):
    """Concatenate datasets for a batched fit: (u, v, families, dataset_offsets,
    subset_offsets (global, sum K + 1), dataset_subset_start (B+1))."""
    u = np.concatenate([d.u for d in datasets])
    v = np.concatenate([d.v for d in datasets])
    fam = np.array([d.family for d in datasets], dtype=np.int32)
    dofs = np.concatenate([[0], np.cumsum([d.n for d in datasets])]).astype(np.int64)
    sub = [np.array([0], dtype=np.int64)]
    starts = [0]
    for i, d in enumerate(datasets):
        sub.append(d.offsets[1:] + dofs[i])
        starts.append(starts[-1] + d.K)
    return u, v, fam, dofs, np.concatenate(sub).astype(np.int64), np.array(starts, dtype=np.int64)
