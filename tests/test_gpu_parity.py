"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars: ranks bit-exact; theta within 1e-9 relative on the FP64 path and 1e-5
on the FP32-compensated path (relative to max(|theta|, 0.05), so that fits at
independence, theta ~ 0, are held to the same absolute scale); statuses equal;
the combined estimate (Eq. 15) to the theta bar.  The variance is compared
where it is defined (status OK or BOUNDARY) within 1e-8 relative on the FP64
path for m >= 16 and 2e-4 on the FP32C path for m >= 64: on tinier subsets
the sandwich's nu^2 is a small difference of large per-point terms, which
FP32 per-point arithmetic cannot resolve.
"""
import os

import numpy as np
import pytest

import copula_synth as cs
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1609_05530_gb300 as cg  # noqa: E402

THETA_TOL = {"f64": 1e-9, "f32c": 1e-5}
VAR_TOL = {"f64": 1e-8, "f32c": 2e-4}
VAR_MIN_M = {"f64": 16, "f32c": 64}
NCPU = os.cpu_count() or 1


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def theta_err(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), 0.05)


def check_fit(u, v, off, fam, prec, weight="invvar", label=""):
    r = cg.fit(dev(u), dev(v), off, fam, prec, weight)
    torch.cuda.synchronize()
    o = oracle.fit(fam, u, v, off, weight=cg.WEIGHTS[weight], nthreads=NCPU)
    th, var, st = r.theta.cpu().numpy(), r.var.cpu().numpy(), r.status.cpu().numpy()
    ok = o["status"] != oracle.DEGENERATE
    assert np.array_equal(st, o["status"]), (label, st, o["status"])
    e = theta_err(th[ok], o["theta"][ok])
    assert e.max() <= THETA_TOL[prec], (label, prec, e.max(), np.argmax(e))
    m = np.diff(np.asarray(off))
    vok = ((o["status"] == oracle.OK) | (o["status"] == oracle.BOUNDARY)) & (m >= VAR_MIN_M[prec])
    if vok.any():
        ve = np.abs(var[vok] - o["var"][vok]) / np.abs(o["var"][vok])
        assert ve.max() <= VAR_TOL[prec], (label, prec, ve.max(), np.argmax(ve))
    ce = theta_err(r.combined.item(), o["combined"])
    assert ce <= THETA_TOL[prec], (label, prec, ce)
    return r, o


# ---------------------------------------------------------------------------
# Eq. 12: ranks
# ---------------------------------------------------------------------------

RAGGED = [2, 3, 31, 32, 33, 100, 1000, 1537, 4097, 6145, cg.MAX_SUBSET]


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_ranks_bit_exact(dtype):
    g = np.random.default_rng(1)
    sizes = RAGGED[:-1] + [cg.MAX_SUBSET if dtype == np.float32 else cg.MAX_SUBSET_F64] + [500] * 5
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(off[-1])
    x = g.random(n).astype(dtype)
    x[g.integers(0, n, n // 5)] = x[g.integers(0, n, n // 5)]  # many exact ties
    x[5:9] = -0.0
    x[9:13] = 0.0                                  # -0.0 ties +0.0 (ordinal by row)
    x[2000:2100] = dtype(0.25)                     # a run of ties
    x[n - 50:] = -np.abs(x[n - 50:])               # negatives
    r = cg.ranks(dev(x), off).cpu().numpy()
    assert np.array_equal(r, oracle.ranks(x, off))


def test_ranks_value_buckets_and_their_fallback():
    """Ranks through both orderings of the shared-memory path, bit-exact: the
    value-bucket ranking (spread-out values) and the radix sort it falls back
    to (a crowded bucket, an infinite or overflowing range, denormals, all
    equal), in one call, in subsets of every launch bucket."""
    g = np.random.default_rng(11)
    parts = [
        g.random(10_000),                                   # uniform margins
        g.standard_normal(6_000),                           # normal margins
        g.exponential(size=9_000),                          # skewed margins
        g.standard_cauchy(8_000),                           # heavy tails: a crowded bucket
        (g.random(7_000) - 0.5) * 6e38,                     # range overflows FP32
        g.random(3_000) * 1e-40,                            # denormals
        np.round(g.random(12_000) * 40) / 40,               # 41 distinct values
        np.arange(4_096) / 4_096.0,                         # values on bucket edges
        np.concatenate([g.random(2_000), 1e6 + g.random(2_000)]),  # two far clusters
        np.concatenate([np.full(1_500, 0.5), [0.7]]),       # all equal but one
        np.where(g.random(900) < 0.5, -0.0, 0.0) + (g.random(900) < 0.3),
        g.random(2), g.random(3), g.random(8), g.random(33),
        -g.random(20_000) * 1e-3 + 0.25,                    # narrow range, negatives offset
        g.permutation(cg.MAX_SUBSET).astype(np.float64),    # exact integers, largest subset
    ]
    x = np.concatenate(parts).astype(np.float32)
    x[g.integers(0, x.shape[0], 2_000)] = x[g.integers(0, x.shape[0], 2_000)]   # ties across the board
    off = np.concatenate([[0], np.cumsum([p.shape[0] for p in parts])]).astype(np.int64)
    r = cg.ranks(dev(x), off).cpu().numpy()
    assert np.array_equal(r, oracle.ranks(x, off))


def test_ranks_nan_subset_is_zero():
    x = np.random.default_rng(2).random(3000).astype(np.float32)
    x[1500] = np.nan
    off = np.array([0, 1000, 2000, 3000])
    r = cg.ranks(dev(x), off).cpu().numpy()
    assert np.all(r[1000:2000] == 0)
    good = np.r_[0:1000, 2000:3000]
    assert np.array_equal(r[good], oracle.ranks(np.delete(x, np.s_[1000:2000]), [0, 1000, 2000]))


# ---------------------------------------------------------------------------
# Fits: every family, both precisions, ragged subsets across all launch buckets
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["f64", "f32c"])
@pytest.mark.parametrize("fam,theta", [(0, 0.5), (0, -0.35), (1, 5.0), (1, -2.5), (2, 2.0), (2, 5.0)])
def test_fit_parity_ragged(fam, theta, prec):
    sizes = [2, 3, 5, 31, 33, 100, 1000, 1537, 3000, 6145, 9000, cg.MAX_SUBSET]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    d = cs.make_dataset(fam, theta, int(off[-1]), 1, np.float32, seed=900 + fam * 10 + int(abs(theta) * 7),
                        offsets=off)
    check_fit(d.u, d.v, off, fam, prec, label=f"ragged fam{fam} th{theta}")


@pytest.mark.parametrize("prec", ["f64", "f32c"])
@pytest.mark.parametrize("K", [10, 1])
def test_gaussian_rho05_n1e4_fp64_storage(prec, K):
    """Gaussian rho=0.5, n=10,000 pairs in FP64, K=10 equal subsets (and the
    K=1 full-data fit), equal-weight and inverse-variance combines."""
    d = cs.gaussian_10k(np.float64, K=K)
    check_fit(d.u, d.v, d.offsets, 0, prec, "invvar", "gauss10k")
    check_fit(d.u, d.v, d.offsets, 0, prec, "equal", "gauss10k-eq")


@pytest.mark.parametrize("prec", ["f64", "f32c"])
def test_frank_theta5_n1e6_k100(prec):
    """Frank theta=5, n=1e6 FP32 pairs, K=100 equal subsets: the full-size
    workload, every subset checked."""
    d = cs.frank_1m()
    check_fit(d.u, d.v, d.offsets, 1, prec, label="frank1m")


@pytest.mark.parametrize("prec", ["f64", "f32c"])
def test_independence_and_weak_dependence(prec):
    # Frank near theta = 0 (series branch), and both signs
    for th, seed in [(0.0, 1), (0.3, 2), (-0.3, 3), (0.04, 4)]:
        d = cs.make_dataset(1, th, 24_000, 6, np.float32, seed=1000 + seed)
        check_fit(d.u, d.v, d.offsets, 1, prec, label=f"frank-indep{th}")


@pytest.mark.parametrize("prec", ["f64", "f32c"])
def test_gumbel_boundary(prec):
    # negatively dependent data: the Gumbel MPL sits on theta = 1
    d = cs.make_dataset(0, -0.5, 4000, 4, np.float32, seed=77)
    r, o = check_fit(d.u, d.v, d.offsets, 2, prec, label="gumbel-boundary")
    assert np.all(r.status.cpu().numpy() == cg.BOUNDARY)
    assert np.all(r.theta.cpu().numpy() == 1.0)


def test_degenerate_subset_is_left_out():
    d = cs.make_dataset(1, 5.0, 3000, 3, np.float32, seed=5)
    u = d.u.copy()
    u[1234] = np.nan
    r = cg.fit(dev(u), dev(d.v), d.offsets, 1, "f64")
    st = r.status.cpu().numpy()
    assert list(st) == [0, cg.DEGENERATE, 0]
    assert np.isnan(r.theta.cpu().numpy()[1])
    o0 = oracle.fit(1, d.u[:1000], d.v[:1000], [0, 1000])
    o2 = oracle.fit(1, d.u[2000:], d.v[2000:], [0, 1000])
    w = np.array([1 / o0["var"][0], 1 / o2["var"][0]])
    comb = (w[0] * o0["theta"][0] + w[1] * o2["theta"][0]) / w.sum()
    assert theta_err(r.combined.item(), comb) <= 1e-9


@pytest.mark.parametrize("weight", ["fisher", "equal"])
def test_weight_modes(weight):
    d = cs.make_dataset(2, 2.0, 30_000, 7, np.float32, seed=8)
    check_fit(d.u, d.v, d.offsets, 2, "f64", weight, label=weight)


@pytest.mark.parametrize("prec", ["f64", "f32c"])
@pytest.mark.parametrize("fam,theta", [(0, 0.6), (1, 4.0), (1, -3.0), (1, 0.01), (2, 1.8)])
def test_loglik_pass_parity(fam, theta, prec):
    d = cs.make_dataset(fam, theta, 12_000, 3, np.float32, seed=44)
    ths = np.array([theta * 0.9 + (0.0 if fam else 0.0), theta, theta * 1.1 if fam != 2 else theta + 0.2])
    if fam == 0:
        ths = np.clip(ths, -0.95, 0.95)
    if fam == 2:
        ths = np.maximum(ths, 1.0)
    l, g, h = (x.cpu().numpy() for x in cg.loglik(dev(d.u), dev(d.v), d.offsets, fam, ths, prec))
    tol = 1e-10 if prec == "f64" else 2e-6
    for k in range(3):
        lo, hi = d.offsets[k], d.offsets[k + 1]
        ru = oracle.ranks(d.u[lo:hi], [0, hi - lo])
        rv = oracle.ranks(d.v[lo:hi], [0, hi - lo])
        ol, og, oh = oracle.loglik(fam, ths[k], ru, rv)
        m = hi - lo
        # scale: per-point magnitude times m
        assert abs(l[k] - ol) <= tol * max(abs(ol), m), (k, l[k], ol)
        assert abs(g[k] - og) <= tol * max(abs(oh), m), (k, g[k], og)
        assert abs(h[k] - oh) <= tol * max(abs(oh), m), (k, h[k], oh)


# ---------------------------------------------------------------------------
# Batching and the host-buffer entry point
# ---------------------------------------------------------------------------

def _mixed(B=24, seed=5):
    g = np.random.default_rng(seed)
    ds = []
    for b in range(B):
        fam = int(g.integers(0, 3))
        tau = float(g.uniform(0.1, 0.8))
        n = int(np.exp(g.uniform(np.log(300), np.log(60_000))))
        K = max(1, n // 10_000)
        ds.append(cs.make_dataset(fam, cs.theta_of_tau(fam, tau), n, K, np.float32, seed=seed * 1000 + b))
    return ds


@pytest.mark.parametrize("prec", ["f64", "f32c"])
def test_batch_matches_oracle_and_single_fits(prec):
    ds = _mixed()
    u, v, fam, dofs, soff, dss = cs.pack_batch(ds)
    r = cg.fit_batch(dev(u), dev(v), fam, dofs, soff, dss, prec)
    th, var, comb = r.theta.cpu().numpy(), r.var.cpu().numpy(), r.combined.cpu().numpy()
    for b, d in enumerate(ds):
        sl = slice(dss[b], dss[b + 1])
        o = oracle.fit(d.family, d.u, d.v, d.offsets, nthreads=NCPU)
        assert theta_err(th[sl], o["theta"]).max() <= THETA_TOL[prec], b
        assert theta_err(comb[b], o["combined"]) <= THETA_TOL[prec], b
        # the same subset gives the same bits alone and in the mix
        s = cg.fit(dev(d.u), dev(d.v), d.offsets, d.family, prec)
        assert np.array_equal(s.theta.cpu().numpy(), th[sl]), b
        assert np.array_equal(s.var.cpu().numpy(), var[sl]), b


def test_batch_permutation_invariance():
    ds = _mixed(12, seed=9)
    a = cg.fit_batch(*(lambda p: (dev(p[0]), dev(p[1]), p[2], p[3], p[4], p[5]))(cs.pack_batch(ds)), "f32c")
    perm = list(reversed(range(len(ds))))
    b = cg.fit_batch(*(lambda p: (dev(p[0]), dev(p[1]), p[2], p[3], p[4], p[5]))(cs.pack_batch([ds[i] for i in perm])),
                     "f32c")
    ca, cb = a.combined.cpu().numpy(), b.combined.cpu().numpy()
    assert np.array_equal(ca[perm], cb)


@pytest.mark.parametrize("pinned", [False, True])
@pytest.mark.parametrize("prec", ["f64", "f32c"])
def test_fit_host_matches_device_fit(prec, pinned):
    """Pageable host inputs are copied into the workspace first; pinned ones
    are read by the kernel over the host link.  Same bits either way."""
    d = cs.make_dataset(1, 5.0, 50_000, 5, np.float32, seed=3)
    u, v = d.u, d.v
    if pinned:
        u, v = torch.from_numpy(d.u).pin_memory(), torch.from_numpy(d.v).pin_memory()
    th, var, st, comb = cg.fit_host(u, v, d.offsets, 1, prec)
    r = cg.fit(dev(d.u), dev(d.v), d.offsets, 1, prec)
    assert np.array_equal(th, r.theta.cpu().numpy())
    assert np.array_equal(var, r.var.cpu().numpy())
    assert np.array_equal(st, r.status.cpu().numpy())
    assert comb[0] == r.combined.item()


@pytest.mark.parametrize("prec", ["f64", "f32c"])
def test_fit_host_pinned_with_streaming_subsets(prec):
    """A pinned request with a subset above the shared-memory size takes the
    copy path (the streaming kernels read their inputs several times)."""
    off = np.array([0, 3000, 3000 + 45_000, 50_000], np.int64)
    d = cs.make_dataset(2, 2.0, 50_000, 1, np.float32, seed=33, offsets=off)
    u, v = torch.from_numpy(d.u).pin_memory(), torch.from_numpy(d.v).pin_memory()
    th, var, st, comb = cg.fit_host(u, v, off, 2, prec)
    r = cg.fit(dev(d.u), dev(d.v), off, 2, prec)
    assert np.array_equal(th, r.theta.cpu().numpy())
    assert np.array_equal(var, r.var.cpu().numpy())
    assert comb[0] == r.combined.item()


def test_repeat_calls_are_bitwise_stable():
    d = cs.make_dataset(2, 2.0, 40_000, 4, np.float32, seed=12)
    a = cg.fit(dev(d.u), dev(d.v), d.offsets, 2, "f32c")
    b = cg.fit(dev(d.u), dev(d.v), d.offsets, 2, "f32c")
    assert np.array_equal(a.theta.cpu().numpy(), b.theta.cpu().numpy())
    assert np.array_equal(a.var.cpu().numpy(), b.var.cpu().numpy())


def test_argument_errors_are_reported():
    d = cs.make_dataset(1, 5.0, 1000, 1, np.float32, seed=3)
    with pytest.raises(cg.CopulaError):
        cg.fit(dev(d.u), dev(d.v), [0, 1, 1000], 1)
    with pytest.raises(cg.CopulaError):
        cg.fit(dev(d.u), dev(d.v), [0, 999], 1)
    with pytest.raises(cg.CopulaError):
        cg.fit(dev(d.u), dev(d.v), [0, 1000], 7)


@pytest.mark.parametrize("prec", ["f64", "f32c"])
@pytest.mark.parametrize("fam,theta", [(1, 5.0), (1, -2.0), (2, 2.0), (2, 6.0)])
def test_newton_stops_after_a_few_passes(fam, theta, prec):
    """Newton from the Spearman start converges quadratically: once a step
    falls below the tolerance (at the root it rounds onto theta itself) the
    search stops, instead of treating the sub-ulp step as a bracket failure
    and bisecting from a search cap.  Both paths: shared-memory subsets and
    streaming ones."""
    off = np.concatenate([[0], np.cumsum([5000] * 6 + [60_000])]).astype(np.int64)
    d = cs.make_dataset(fam, theta, int(off[-1]), 1, np.float32, seed=321, offsets=off)
    r, dg = cg.fit_ex(dev(d.u), dev(d.v), off, fam, prec)
    it = dg.iters.cpu().numpy()
    assert np.all(r.status.cpu().numpy() == cg.OK)
    assert it.max() <= 7, it
    o = oracle.fit(fam, d.u, d.v, off, nthreads=NCPU)
    assert theta_err(r.theta.cpu().numpy(), o["theta"]).max() <= THETA_TOL[prec]


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_ranks_infinities_and_all_equal_subsets(dtype):
    """+inf ranks last and -inf first (ordinal among equals), a subset of one
    repeated value ranks in row order, on the shared-memory path."""
    g = np.random.default_rng(31)
    sizes = [1000, 2048, 777, 5000]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    x = g.standard_normal(int(off[-1])).astype(dtype)
    x[g.integers(0, 1000, 50)] = np.inf
    x[g.integers(0, 1000, 50)] = -np.inf
    x[off[1]:off[2]] = dtype(3.25)                    # all equal
    x[off[2]:off[2] + 10] = -0.0
    x[off[2] + 10:off[2] + 20] = 0.0
    x[off[3]:off[4]] = np.sort(x[off[3]:off[4]])[::-1]  # descending
    r = cg.ranks(dev(x), off).cpu().numpy()
    assert np.array_equal(r, oracle.ranks(x, off))
    assert np.array_equal(r[off[1]:off[2]], np.arange(1, sizes[1] + 1))


def test_plan_cache_follows_partition_family_and_block_changes():
    """A context reuses its last plan only for the same arguments: fits that
    alternate between partitions, families and block tables on one context
    equal fits on fresh contexts, bit for bit."""
    d = cs.make_dataset(1, 4.0, 60_000, 6, np.float32, seed=1300)
    u, v = dev(d.u), dev(d.v)
    offs = [d.offsets, cs.equal_offsets(60_000, 5), d.offsets]
    ctx = cg.Context()
    for i, (off, fam) in enumerate([(offs[0], 1), (offs[1], 1), (offs[2], 1), (offs[0], 2), (offs[0], 1)]):
        got = cg.fit(u, v, off, fam, "f32c", ctx=ctx)
        ref = cg.fit(u, v, off, fam, "f32c", ctx=cg.Context())
        assert torch.equal(got.theta, ref.theta) and torch.equal(got.combined, ref.combined), i
    cg.set_blocks([(20480, 256)], ctx)
    got = cg.fit(u, v, offs[0], 1, "f32c", ctx=ctx)
    c2 = cg.Context()
    cg.set_blocks([(20480, 256)], c2)
    ref = cg.fit(u, v, offs[0], 1, "f32c", ctx=c2)
    assert torch.equal(got.theta, ref.theta)
    # the same plan again on other data: the cached plan's upload image is
    # copied as it stands, the results are the new data's
    d2 = cs.make_dataset(1, -2.0, 60_000, 6, np.float32, seed=1301, offsets=offs[0])
    u2, v2 = dev(d2.u), dev(d2.v)
    for uu, vv in ((u2, v2), (u, v), (u2, v2)):
        got = cg.fit(uu, vv, offs[0], 1, "f32c", ctx=ctx)
        ref = cg.fit(uu, vv, offs[0], 1, "f32c", ctx=c2)
        assert torch.equal(got.theta, ref.theta) and torch.equal(got.var, ref.var)
