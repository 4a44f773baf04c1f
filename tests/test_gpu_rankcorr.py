"""copula_rank_corr: Kendall's tau and Spearman's rho of every subset, against
the oracle's definitions (every pair compared; 1 - 6 sum d^2 / (m(m^2-1))),
bit for bit: both are integer counts followed by one FP64 division in the
same order.  Sizes span every launch bucket and the shared-memory limit;
ties, -0.0/+0.0, all-equal, sorted and reversed subsets, NaN, FP64 storage,
and streaming-size subsets up to the size limit are covered."""
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


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def oracle_corr(u, v, off):
    ru, rv = oracle.ranks(u, off), oracle.ranks(v, off)
    tau = np.array([oracle.kendall_tau(ru[a:b], rv[a:b]) for a, b in zip(off[:-1], off[1:])])
    rho = np.array([oracle.spearman_rho(ru[a:b], rv[a:b]) for a, b in zip(off[:-1], off[1:])])
    return tau, rho


def offsets(sizes):
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


@pytest.mark.parametrize("fam,theta", [(1, 5.0), (2, 2.0), (0, -0.4)])
def test_rank_corr_bit_exact_across_buckets(fam, theta):
    sizes = [2, 3, 100, 1536, 1537, 6144, 6145, 20_480, 777]
    off = offsets(sizes)
    d = cs.make_dataset(fam, theta, int(off[-1]), 1, np.float32, seed=6100 + fam, offsets=off)
    u = np.round(d.u * 4000).astype(np.float32) / 4000  # ties: ranks by row index among equals
    tau, rho = (x.cpu().numpy() for x in cg.rank_corr(dev(u), dev(d.v), off))
    ot, orho = oracle_corr(u, d.v, off)
    assert np.array_equal(tau, ot), np.abs(tau - ot).max()
    assert np.array_equal(rho, orho), np.abs(rho - orho).max()


def test_rank_corr_fp64_storage_and_special_subsets():
    sizes = [500, 15_000, 1000, 1000, 64, 300]
    off = offsets(sizes)
    d = cs.make_dataset(1, -3.0, int(off[-1]), 1, np.float64, seed=6200, offsets=off)
    u, v = d.u.copy(), d.v.copy()
    a, b = off[2], off[3]
    u[a:b] = np.sort(u[a:b])
    v[a:b] = np.sort(v[a:b])                # concordant: tau = rho = 1
    a, b = off[3], off[4]
    u[a:b] = np.sort(u[a:b])
    v[a:b] = np.sort(v[a:b])[::-1]          # discordant: tau = rho = -1
    a, b = off[4], off[5]
    u[a:b] = 2.5                            # all equal: ranks in row order
    v[a:b] = 0.0
    v[a:a + 32] = -0.0                      # -0.0 equals +0.0
    tau, rho = (x.cpu().numpy() for x in cg.rank_corr(dev(u), dev(v), off))
    ot, orho = oracle_corr(u, v, off)
    assert np.array_equal(tau, ot) and np.array_equal(rho, orho)
    assert tau[2] == 1.0 and rho[2] == 1.0 and tau[3] == -1.0 and rho[3] == -1.0
    assert tau[4] == 1.0 and rho[4] == 1.0


def test_rank_corr_nan_subset_only():
    off = offsets([1000, 2000, 1500])
    d = cs.make_dataset(2, 3.0, int(off[-1]), 1, np.float32, seed=6300, offsets=off)
    v = d.v.copy()
    v[off[1] + 17] = np.nan
    tau, rho = (x.cpu().numpy() for x in cg.rank_corr(dev(d.u), dev(v), off))
    assert np.isnan(tau[1]) and np.isnan(rho[1])
    keep = [0, 2]
    sub = offsets([1000, 1500])
    u2 = np.concatenate([d.u[:1000], d.u[3000:]])
    v2 = np.concatenate([v[:1000], v[3000:]])
    ot, orho = oracle_corr(u2, v2, sub)
    assert np.array_equal(tau[keep], ot) and np.array_equal(rho[keep], orho)


def test_rank_corr_streaming_sizes_bit_exact():
    """Subsets above the shared-memory limit (ranked by the sample sort, their
    inversions counted chunk by chunk: 2, 3 and 4 chunks of 16,384 with ragged
    ends), with ties and negatives, beside small ones, against the oracle's
    every-pair tau and its rho, bit for bit; and a NaN subset of that size."""
    off = offsets([1000, cg.MAX_SUBSET + 1, 40_000, 33_000, 50_001])
    d = cs.make_dataset(1, 3.0, int(off[-1]), 1, np.float32, seed=6400, offsets=off)
    u, v = d.u.copy(), d.v.copy()
    g = np.random.default_rng(5)
    u[g.integers(0, u.shape[0], 3000)] = u[g.integers(0, u.shape[0], 3000)]   # ties
    v[off[3]:off[4]] = -v[off[3]:off[4]]                                      # negative dependence
    tau, rho = cg.rank_corr(dev(u), dev(v), off)
    ot, orr = oracle_corr(u, v, off)
    assert np.array_equal(tau.cpu().numpy(), ot)
    assert np.array_equal(rho.cpu().numpy(), orr)
    u[off[2] + 777] = np.nan
    tau, rho = cg.rank_corr(dev(u), dev(v), off)
    t, r = tau.cpu().numpy(), rho.cpu().numpy()
    assert np.isnan(t[2]) and np.isnan(r[2])
    keep = [0, 1, 3, 4]
    assert np.array_equal(t[keep], ot[keep]) and np.array_equal(r[keep], orr[keep])


def test_rank_corr_at_the_streaming_limit():
    """One subset of the largest streaming size (3,145,728 rows, 192 chunks):
    tau against the oracle's merge count (exact: integer counts, one
    division).  rho: sum d^2 reaches ~1e19 here, beyond 2^53, where the
    oracle's FP64 running sum rounds (relative error up to ~m eps = 3.5e-10
    of D, ~1e-10 in rho); the kernel's 128-bit count is exact, so it is
    compared bit for bit with the exact integer sum taken here, and with the
    oracle to 1e-10."""
    m = cg.MAX_SUBSET_STREAM
    g = torch.Generator(device="cuda")
    g.manual_seed(6450)
    u, v = dsyn.sample(2, 2.0, m, g)
    u, v = u.float(), v.float()
    off = np.array([0, m], dtype=np.int64)
    tau, rho = cg.rank_corr(u, v, off)
    hu, hv = u.cpu().numpy(), v.cpu().numpy()
    ru, rv = oracle.ranks(hu, off), oracle.ranks(hv, off)
    assert tau.item() == oracle.kendall_tau_merge(ru, rv)
    d = ru.astype(np.int64) - rv.astype(np.int64)
    D = sum(int(np.sum(d[i:i + 100_000] ** 2)) for i in range(0, m, 100_000))   # exact (Python integers)
    md = float(m)
    assert rho.item() == 1.0 - 6.0 * float(D) / (md * (md * md - 1.0))
    assert abs(rho.item() - oracle.spearman_rho(ru, rv)) <= 1e-10


def test_rank_corr_inverts_to_the_generating_parameter():
    """Subsets at the shared-memory limit (20,480 rows) of a Frank theta = 5
    sample: their taus, inverted by the oracle's map, average within five
    standard errors of theta (about 0.005 in tau per subset, over 8)."""
    K, m = 8, 20_480
    d = cs.make_dataset(1, 5.0, K * m, K, np.float32, seed=6500)
    tau, _ = cg.rank_corr(dev(d.u), dev(d.v), d.offsets)
    th = np.mean([oracle.theta_from_tau(1, t)[0] for t in tau.cpu().numpy()])
    slope = 0.02 / (oracle.tau_of_theta(1, 5.01) - oracle.tau_of_theta(1, 4.99))
    assert abs(th - 5.0) < 5 * 0.005 / np.sqrt(K) * slope


# ---------------------------------------------------------------------------
# copula_theta_from_rank_corr: the inversion itself, against the oracle's
# population maps and its bisection (theta within 1e-9 relative to
# max(|theta|, 0.05), equal statuses); Gumbel's rho_S map is steep in theta at
# large theta (d theta / d rho_S ~ 3e4 at theta = 45), so there the GPU theta
# is checked through the oracle's map, in rho_S, to 1e-10.
# ---------------------------------------------------------------------------

R_GRID = np.concatenate([np.linspace(-0.98, 0.98, 99), [0.0, 1e-3, -1e-3, 0.4999, 0.9999, -0.9999, 1.0, -1.0]])


def _oracle_inverse(fam, which, r):
    f = oracle.theta_from_tau if which == "tau" else oracle.theta_from_rho_s
    out = [f(fam, float(x)) for x in r]
    return np.array([o[0] for o in out]), np.array([o[1] for o in out])


@pytest.mark.parametrize("which", ["tau", "rho"])
@pytest.mark.parametrize("fam", [0, 1, 2])
def test_theta_from_rank_corr_matches_oracle(fam, which):
    # (the oracle's Gumbel rho_S inverse bisects on a 2-D quadrature: a
    # coarser grid keeps it to seconds)
    r = np.concatenate([R_GRID[:99:4], R_GRID[99:]]) if (fam == 2 and which == "rho") else R_GRID
    th, st = cg.theta_from_rank_corr(dev(r), fam, which)
    th, st = th.cpu().numpy(), st.cpu().numpy()
    oth, ost = _oracle_inverse(fam, which, r)
    assert np.array_equal(st, ost), (fam, which, r[st != ost], st[st != ost], ost[st != ost])
    ok = np.isfinite(oth)
    if fam == 2 and which == "rho":
        inner = ok & (st == oracle.OK)
        back = np.array([oracle.rho_s_of_theta(2, float(t)) for t in th[inner]])
        assert np.abs(back - r[inner]).max() <= 1e-10
        e = np.abs(th[ok] - oth[ok]) / np.maximum(np.abs(oth[ok]), 0.05)
        assert e.max() <= 1e-6
    else:
        e = np.abs(th[ok] - oth[ok]) / np.maximum(np.abs(oth[ok]), 0.05)
        assert e.max() <= 1e-9, (fam, which, e.max(), r[np.argmax(e)])


def test_theta_from_rank_corr_special_values():
    r = dev(np.array([np.nan, 1.5, -1.2, 0.0, -0.3]))
    th, st = cg.theta_from_rank_corr(r, 1, "tau")
    st = st.cpu().numpy()
    assert list(st[:3]) == [cg.DEGENERATE] * 3 and np.isnan(th.cpu().numpy()[:3]).all()
    assert st[3] == cg.OK and th.cpu().numpy()[3] == 0.0
    th, st = cg.theta_from_rank_corr(dev(np.array([-0.3, 0.0])), 2, "rho")
    assert (st.cpu().numpy() == cg.BOUNDARY).all() and (th.cpu().numpy() == 1.0).all()


@pytest.mark.parametrize("fam,theta", [(1, 5.0), (1, -3.0), (2, 2.0), (0, 0.5)])
def test_inversion_estimator_on_data(fam, theta):
    """The whole inversion estimator per subset -- sample tau and rho_S of the
    subset's ranks (Eq. 12), then the inverse map -- against the oracle's
    statistics and inverse on the same subsets."""
    sizes = [500, 3000, 9000, 20_000]
    off = offsets(sizes)
    d = cs.make_dataset(fam, theta, int(off[-1]), 1, np.float32, seed=6600 + fam, offsets=off)
    tau, rho = cg.rank_corr(dev(d.u), dev(d.v), off)
    ot, orr = oracle_corr(d.u, d.v, off)
    for which, val, oval in (("tau", tau, ot), ("rho", rho, orr)):
        th, st = cg.theta_from_rank_corr(val, fam, which)
        oth, ost = _oracle_inverse(fam, which, oval)
        assert np.array_equal(st.cpu().numpy(), ost)
        e = np.abs(th.cpu().numpy() - oth) / np.maximum(np.abs(oth), 0.05)
        assert e.max() <= (1e-6 if (fam == 2 and which == "rho") else 1e-9), (which, e.max())
