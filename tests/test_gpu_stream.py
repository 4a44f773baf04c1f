"""Parity of the streaming path -- subsets larger than one thread block's
shared-memory sort, ranked by a multi-block sample sort and fitted by one
cooperative kernel -- with the FP64 CPU oracle.

Same bars as the shared-memory path: ranks bit-exact (ties by row, -0.0 ==
+0.0, NaN subsets all zero); theta within 1e-9 (FP64) / 1e-5 (FP32C) of the
oracle's; statuses equal; variances where defined; Eq. 15 on top.  Subset
sizes straddle the single-block limit, chunk boundaries (16,384 rows) and leave
ragged tails, mixed in one call with small subsets.  The Gumbel n = 1e8,
K = 1000 lognormal-size workload is fitted in full and checked on sampled
subsets (the largest among them) and through the oracle's combine.
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
from copula_synth import device as dsyn  # noqa: E402

THETA_TOL = {"f64": 1e-9, "f32c": 1e-5}
VAR_TOL = {"f64": 1e-8, "f32c": 2e-4}
NCPU = os.cpu_count() or 1

BIG32 = [cg.MAX_SUBSET + 1, 65_537, 150_000]      # 2, 5 (last chunk of 1 row) and 10 chunks of 16,384
BIG64 = [cg.MAX_SUBSET_F64 + 1, 65_537, 100_003]


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def theta_err(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), 0.05)


def offsets(sizes):
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def check_fit(u, v, off, fam, prec, label=""):
    r = cg.fit(dev(u), dev(v), off, fam, prec)
    torch.cuda.synchronize()
    o = oracle.fit(fam, u, v, off, nthreads=NCPU)
    th, var, st = r.theta.cpu().numpy(), r.var.cpu().numpy(), r.status.cpu().numpy()
    assert np.array_equal(st, o["status"]), (label, st, o["status"])
    ok = o["status"] != oracle.DEGENERATE
    e = theta_err(th[ok], o["theta"][ok])
    assert e.max() <= THETA_TOL[prec], (label, prec, e.max(), np.argmax(e))
    vok = (o["status"] == oracle.OK) | (o["status"] == oracle.BOUNDARY)
    if vok.any():
        ve = np.abs(var[vok] - o["var"][vok]) / np.abs(o["var"][vok])
        assert ve.max() <= VAR_TOL[prec], (label, prec, ve.max(), np.argmax(ve))
    assert theta_err(r.combined.item(), o["combined"]) <= THETA_TOL[prec], label
    return r, o


# ---------------------------------------------------------------------------
# Eq. 12 on the streaming path: ranks
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_stream_ranks_bit_exact(dtype):
    g = np.random.default_rng(11)
    big = BIG32 if dtype == np.float32 else BIG64
    sizes = [500] + big + [1000, 120_000, 90_000, 70_000, 3]
    off = offsets(sizes)
    n = int(off[-1])
    x = g.random(n).astype(dtype)
    x[g.integers(0, n, n // 5)] = x[g.integers(0, n, n // 5)]  # many exact ties
    s1 = off[1]
    x[s1 + 5:s1 + 9] = -0.0
    x[s1 + 9:s1 + 13] = 0.0                                      # -0.0 ties +0.0
    x[s1 + 2000:s1 + 12_000] = dtype(0.25)                       # a run of ties longer than a bucket
    k = len(big) + 2                                             # the 120k subset: all equal
    x[off[k]:off[k + 1]] = dtype(0.5)
    k += 1                                                       # 90k: sorted ascending
    x[off[k]:off[k + 1]] = np.sort(x[off[k]:off[k + 1]])
    k += 1                                                       # 70k: periodic with the sample stride
    x[off[k]:off[k + 1]] = (np.arange(off[k + 1] - off[k]) % 273).astype(dtype)
    x[n - 50:] = -np.abs(x[n - 50:])
    r = cg.ranks(dev(x), off).cpu().numpy()
    assert np.array_equal(r, oracle.ranks(x, off))


def test_stream_ranks_nan_subset_is_zero():
    x = np.random.default_rng(2).random(3 * 30_000).astype(np.float32)
    x[45_000] = np.nan
    off = np.array([0, 30_000, 60_000, 90_000])
    r = cg.ranks(dev(x), off).cpu().numpy()
    assert np.all(r[30_000:60_000] == 0)
    good = np.r_[0:30_000, 60_000:90_000]
    assert np.array_equal(r[good], oracle.ranks(np.delete(x, np.s_[30_000:60_000]), [0, 30_000, 60_000]))


# ---------------------------------------------------------------------------
# Fits: every family, both precisions, large subsets mixed with small ones
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["f64", "f32c"])
@pytest.mark.parametrize("fam,theta", [(0, 0.5), (0, -0.35), (1, 5.0), (1, -2.5), (1, 0.3), (2, 2.0), (2, 5.0)])
def test_stream_fit_parity(fam, theta, prec):
    sizes = [700] + BIG32 + [5000]
    off = offsets(sizes)
    d = cs.make_dataset(fam, theta, int(off[-1]), 1, np.float32, seed=4100 + fam * 10 + int(abs(theta) * 7),
                        offsets=off)
    check_fit(d.u, d.v, off, fam, prec, label=f"stream fam{fam} th{theta}")


@pytest.mark.parametrize("prec", ["f64", "f32c"])
def test_stream_fit_kernel_barrier_stamps(prec):
    """A timed call records the streaming fit kernel's barrier releases: in
    order, within the kernel's span, one per chunk sweep and Newton step
    (two sweeps before the passes in FP32, three in FP64 plus three around
    the FP32 start search; then the variance sweeps)."""
    from bench import FIT_VARIANCE_BARRIERS
    off = offsets([700] + BIG32)
    d = cs.make_dataset(2, 2.0, int(off[-1]), 1, np.float32, seed=4150, offsets=off)
    ctx = cg.Context()
    u, v = torch.from_numpy(d.u).cuda(), torch.from_numpy(d.v).cuda()
    o = cg.make_opts(prec)
    ctx.set_timing(True)
    cg.fit_ex(u, v, off, 2, ctx=ctx, opts=o)
    fit_ms = ctx.stage_ms()[3]
    t = ctx.stream_stamps()
    ctx.set_timing(False)
    assert np.all(np.diff(t) >= 0) and t[0] >= 0 and t[-1] <= fit_ms * 1e6 + 1e4
    fixed = (2 if prec == "f32c" else 3 + 3) + FIT_VARIANCE_BARRIERS
    assert len(t) >= fixed + 2 and (len(t) - fixed) % 2 == 0
    ctx.set_timing(True)
    cg.fit(u[:700], v[:700], np.array([0, 700]), 2, ctx=ctx, opts=o)  # no streaming subset
    with pytest.raises(cg.CopulaError):
        ctx.stream_stamps()
    ctx.set_timing(False)
    ctx.close()


@pytest.mark.parametrize("prec", ["f64", "f32c"])
def test_stream_fit_fp64_storage(prec):
    off = offsets([300] + BIG64)
    d = cs.make_dataset(1, 4.0, int(off[-1]), 1, np.float64, seed=4200, offsets=off)
    check_fit(d.u, d.v, off, 1, prec, label="stream f64 storage")


@pytest.mark.parametrize("prec", ["f64", "f32c"])
def test_stream_gumbel_boundary_and_degenerate(prec):
    off = offsets([30_000, 40_000, 25_000])
    d = cs.make_dataset(0, -0.5, int(off[-1]), 1, np.float32, seed=4300, offsets=off)
    u = d.u.copy()
    u[off[1] + 777] = np.nan
    r = cg.fit(dev(u), dev(d.v), off, 2, prec)
    st = r.status.cpu().numpy()
    assert list(st) == [cg.BOUNDARY, cg.DEGENERATE, cg.BOUNDARY]
    th = r.theta.cpu().numpy()
    assert th[0] == 1.0 and np.isnan(th[1]) and th[2] == 1.0


@pytest.mark.parametrize("prec", ["f64", "f32c"])
@pytest.mark.parametrize("fam,theta", [(0, 0.6), (1, 4.0), (1, -3.0), (1, 0.01), (2, 1.8)])
def test_stream_loglik_parity(fam, theta, prec):
    off = offsets([25_000, 40_961])
    d = cs.make_dataset(fam, theta, int(off[-1]), 1, np.float32, seed=4400, offsets=off)
    ths = np.array([theta, theta * 1.1 if fam != 2 else theta + 0.2])
    if fam == 0:
        ths = np.clip(ths, -0.95, 0.95)
    l, g, h = (x.cpu().numpy() for x in cg.loglik(dev(d.u), dev(d.v), off, fam, ths, prec))
    tol = 1e-10 if prec == "f64" else 2e-6
    for k in range(2):
        lo, hi = off[k], off[k + 1]
        ru = oracle.ranks(d.u[lo:hi], [0, hi - lo])
        rv = oracle.ranks(d.v[lo:hi], [0, hi - lo])
        ol, og, oh = oracle.loglik(fam, ths[k], ru, rv)
        m = hi - lo
        assert abs(l[k] - ol) <= tol * max(abs(ol), m), (k, l[k], ol)
        assert abs(g[k] - og) <= tol * max(abs(oh), m), (k, g[k], og)
        assert abs(h[k] - oh) <= tol * max(abs(oh), m), (k, h[k], oh)


# ---------------------------------------------------------------------------
# Determinism, batching and graph capture
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["f32c", "f64"])
def test_stream_subset_same_bits_alone_and_in_a_batch(prec):
    a = cs.make_dataset(1, 5.0, 60_000, 1, np.float32, seed=4500)
    b = cs.make_dataset(2, 2.0, 90_000, 3, np.float32, seed=4501)
    c = cs.make_dataset(0, 0.4, 45_000, 1, np.float32, seed=4502)
    u, v, fam, dofs, soff, dss = cs.pack_batch([a, b, c])
    r = cg.fit_batch(dev(u), dev(v), fam, dofs, soff, dss, prec)
    th, var = r.theta.cpu().numpy(), r.var.cpu().numpy()
    s = cg.fit(dev(a.u), dev(a.v), a.offsets, 1, prec)
    assert np.array_equal(s.theta.cpu().numpy(), th[:1]) and np.array_equal(s.var.cpu().numpy(), var[:1])
    s = cg.fit(dev(b.u), dev(b.v), b.offsets, 2, prec)
    assert np.array_equal(s.theta.cpu().numpy(), th[1:4]) and np.array_equal(s.var.cpu().numpy(), var[1:4])
    s = cg.fit(dev(c.u), dev(c.v), c.offsets, 0, prec)
    assert np.array_equal(s.theta.cpu().numpy(), th[4:5])
    r2 = cg.fit_batch(dev(u), dev(v), fam, dofs, soff, dss, prec)
    assert np.array_equal(r2.theta.cpu().numpy(), th) and np.array_equal(r2.var.cpu().numpy(), var)


@pytest.mark.parametrize("prec", ["f64", "f32c"])
def test_stream_three_equal_subsets_against_oracle(prec):
    """Three streaming subsets of one dataset (the subsets converge after
    different numbers of passes, so the blocks' loop exits must agree)."""
    d = cs.make_dataset(1, 4.0, 150_000, 3, np.float32, seed=551)
    check_fit(d.u, d.v, d.offsets, 1, prec, label="stream K=3")


@pytest.mark.parametrize("prec", ["f64", "f32c"])
def test_stream_graph_replay_equals_direct(prec):
    ds = [cs.make_dataset(1, 3.0, 70_000, 2, np.float32, seed=4600),
          cs.make_dataset(2, 1.5, 9_000, 3, np.float32, seed=4601),
          cs.make_dataset(0, -0.3, 52_000, 1, np.float32, seed=4602)]
    u, v, fam, dofs, soff, dss = cs.pack_batch(ds)
    plan = cg.BatchPlan(fam, dofs, soff, dss, precision=prec)
    du, dv = dev(u), dev(v)
    g = plan.capture(du, dv)
    g.replay()
    torch.cuda.synchronize()
    direct = cg.fit_batch(dev(u), dev(v), fam, dofs, soff, dss, prec)
    assert torch.equal(plan.theta, direct.theta) and torch.equal(plan.combined, direct.combined)
    # new data in the same buffers
    perm = np.random.default_rng(3).permutation(u.shape[0])
    du.copy_(dev(u[perm]))
    dv.copy_(dev(v[perm]))
    g.replay()
    torch.cuda.synchronize()
    direct2 = cg.fit_batch(du, dv, fam, dofs, soff, dss, prec)
    assert torch.equal(plan.theta, direct2.theta)
    plan.close()


# ---------------------------------------------------------------------------
# Gumbel theta = 2, n = 1e8 FP32 pairs, K = 1000 lognormal(1)-sized subsets
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def gumbel_1e8():
    u, v, off = dsyn.gumbel_lognormal()
    m = np.diff(off)
    # sampled subsets: the largest, the smallest, the largest on the shared-
    # memory path, and four more at random; the oracle fits them once
    order = np.argsort(m)
    pick = {int(order[-1]), int(order[0]), int(np.flatnonzero(m <= cg.MAX_SUBSET)[-1])}
    pick |= set(int(k) for k in np.random.default_rng(7).choice(len(m), 4, replace=False))
    pick = sorted(pick)
    us, vs, sub = [], [], [0]
    for k in pick:
        us.append(u[off[k]:off[k + 1]].cpu().numpy())
        vs.append(v[off[k]:off[k + 1]].cpu().numpy())
        sub.append(sub[-1] + int(m[k]))
    o = oracle.fit(cg.GUMBEL, np.concatenate(us), np.concatenate(vs), np.array(sub, dtype=np.int64), nthreads=NCPU)
    yield u, v, off, pick, o
    del u, v
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", ["f32c", "f64"])
def test_gumbel_1e8_lognormal_sampled_against_oracle(prec, gumbel_1e8):
    u, v, off, pick, o = gumbel_1e8
    r = cg.fit(u, v, off, cg.GUMBEL, prec)
    torch.cuda.synchronize()
    th, var, st = r.theta.cpu().numpy(), r.var.cpu().numpy(), r.status.cpu().numpy()
    assert np.all(st == cg.OK)
    assert np.array_equal(st[pick], o["status"])
    assert theta_err(th[pick], o["theta"]).max() <= THETA_TOL[prec]
    ve = np.abs(var[pick] - o["var"]) / o["var"]
    assert ve.max() <= VAR_TOL[prec]
    # Eq. 15 over all 1000 subsets, by the oracle's combine of the GPU values
    info = np.zeros_like(th)
    assert theta_err(r.combined.item(), oracle.combine(th, var, info, st)) <= 1e-12
    assert abs(r.combined.item() - 2.0) < 1e-3  # sqrt(n)-consistent around the truth


# ---------------------------------------------------------------------------
# The largest subsets the streaming path takes
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dtype,m", [(np.float32, cg.MAX_SUBSET_STREAM), (np.float64, cg.MAX_SUBSET_STREAM_F64)])
def test_stream_ranks_at_the_size_limit(dtype, m):
    g = np.random.default_rng(21)
    x = g.random(m).astype(dtype)
    x[g.integers(0, m, m // 3)] = x[g.integers(0, m, m // 3)]  # ties
    off = np.array([0, m], dtype=np.int64)
    assert np.array_equal(cg.ranks(dev(x), off).cpu().numpy(), oracle.ranks(x, off))


@pytest.fixture(scope="module")
def frank_at_limit():
    m = cg.MAX_SUBSET_STREAM
    off = np.array([0, m], dtype=np.int64)
    d = cs.make_dataset(1, 3.0, m, 1, np.float32, seed=4700, offsets=off)
    return d, off, oracle.ranks(d.u, off), oracle.ranks(d.v, off)


@pytest.mark.parametrize("prec", ["f64", "f32c"])
def test_stream_fit_at_the_size_limit(prec, frank_at_limit):
    """One subset of 3,145,728 rows: the GPU estimate is the root of the
    oracle's score (Eq. 13) -- the oracle's Newton step from it is within the
    theta bar -- and the oracle's sandwich variance there matches."""
    d, off, ru, rv = frank_at_limit
    r = cg.fit(dev(d.u), dev(d.v), off, 1, prec)
    th = float(r.theta.cpu().numpy()[0])
    assert r.status.cpu().numpy()[0] == cg.OK
    _, g, h = oracle.loglik(1, th, ru, rv)
    assert h < 0 and abs(g / h) / max(abs(th), 0.05) <= THETA_TOL[prec]
    var = oracle.var_at(1, th, ru, rv, False)
    assert abs(float(r.var.cpu().numpy()[0]) - var) / var <= VAR_TOL[prec]


@pytest.mark.parametrize("prec", ["f32c", "f64"])
def test_grid_barrier_gives_up_and_leaves_preset_results(prec):
    """The streaming kernel's grid barriers are bounded waits: told to wait for
    one block that does not exist, with a short poll limit, every block gives
    up within milliseconds and returns; the streaming subsets keep their
    preset results (theta and var NaN, status DEGENERATE, the dataset's
    Eq. 15 NaN), the shared-memory subset of the same call is fitted as
    usual, and the context fits correctly again once the limit is lifted."""
    off = offsets([5_000, cg.MAX_SUBSET + 3_000, 40_000])
    d = cs.make_dataset(1, 4.0, int(off[-1]), 1, np.float32, seed=7100, offsets=off)
    ctx = cg.Context()
    u, v = dev(d.u), dev(d.v)
    ctx.set_wait_limit(spins=4096, phantom_arrivals=1)
    r = cg.fit(u, v, off, 1, prec, ctx=ctx)
    torch.cuda.synchronize()
    st, th, var = r.status.cpu().numpy(), r.theta.cpu().numpy(), r.var.cpu().numpy()
    assert st[0] == cg.OK and np.isfinite(th[0])
    assert list(st[1:]) == [cg.DEGENERATE, cg.DEGENERATE]
    assert np.isnan(th[1:]).all() and np.isnan(var[1:]).all()
    assert np.isnan(r.combined.item())
    ctx.set_wait_limit(0, 0)
    r2 = cg.fit(u, v, off, 1, prec, ctx=ctx)
    o = oracle.fit(1, d.u, d.v, off, nthreads=NCPU)
    assert np.array_equal(r2.status.cpu().numpy(), o["status"])
    assert theta_err(r2.theta.cpu().numpy(), o["theta"]).max() <= THETA_TOL[prec]
    assert r2.theta.cpu().numpy()[0] == th[0]    # the shared-memory subset: same bits either way


def _mix32(x):
    """lowbias32 (Wellons), the published integer hash the splitter sampling
    uses to pick a row in each stratum."""
    x ^= x >> 16
    x = (x * 0x7FEB352D) & 0xFFFFFFFF
    x ^= x >> 15
    x = (x * 0x846CA68B) & 0xFFFFFFFF
    x ^= x >> 16
    return x


def _sampled_rows(m, mean):
    nb = max(2, -(-m // mean))
    s = 16 * nb
    return np.array([j * m // s + _mix32(j) % ((j + 1) * m // s - j * m // s) for j in range(s)])


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_stream_ranks_survive_an_overflowing_bucket(dtype):
    """An input built against the splitter sampling: the sampled rows spread
    over [0.1, 0.9], every other row crowded (with ties) into the narrow
    range between the two middle splitters, so that one sample-sort bucket
    holds nearly the whole subset -- far above what one thread block orders
    in shared memory.  That bucket is ranked by direct counting: the ranks
    stay bit-exact, and a fit on such a column matches the oracle."""
    m = 60_000
    mean = 3072 if dtype == np.float32 else 2048
    rows = _sampled_rows(m, mean)
    g = np.random.default_rng(17)
    x = 0.5 + 1e-4 * (g.random(m) - 0.5)
    x[g.integers(0, m, 5000)] = 0.5                           # ties inside the crowded bucket
    x[rows] = np.linspace(0.1, 0.9, rows.shape[0])
    x = x.astype(dtype)
    off = offsets([1000, m, 3000])
    xx = np.concatenate([g.random(1000), x, g.random(3000)]).astype(dtype)
    r = cg.ranks(dev(xx), off).cpu().numpy()
    assert np.array_equal(r, oracle.ranks(xx, off))
    d = cs.make_dataset(1, 3.0, int(off[-1]), 1, dtype, seed=7200, offsets=off)
    for prec in ("f32c", "f64"):
        check_fit(xx, d.v, off, 1, prec, label=f"overflow-{prec}")
