"""Pins of the FP64 CPU oracle against facts outside the oracle itself.

Each pin is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign, a transposed argument, a wrong normaliser) fails at least one:

* the normal quantile against scipy's ``ndtri``;
* ranks against O(m^2) brute-force counting;
* each density against unit integration over [0,1]^2, against the mixed
  derivative of the copula the paper prints (Eq. 10, Eq. 11) and, for the
  Gaussian, against scipy's bivariate normal density (Eq. 7-8);
* the densities against the Spearman's rho / Kendall's tau the paper prints
  for its simulation parameters (Section 2.5, tests/golden);
* score, Hessian and mixed partials against central finite differences;
* the maximiser against the closed-form Gaussian root, against brute force
  on tiny subsets, and against the generating parameter at large n;
* the sandwich variance against its O(m^2) form, the closed form (1-rho^2)^2
  for the Gaussian copula and a Monte-Carlo variance;
* the combine (Eq. 15) against hand arithmetic.
"""
import math
import os

import numpy as np
import pytest
from scipy import special, stats

import copula_synth as cs
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# quadrature helper: tensor Gauss-Legendre on intervals graded towards 0 and 1
# --------------------------------------------------------------------------

def _nodes(nsub=40, order=10):
    edges = (list(np.geomspace(1e-12, 0.02, 20)) + list(np.linspace(0.02, 0.98, nsub)[1:-1]) +
             list(1 - np.geomspace(0.02, 1e-12, 20)))
    edges = np.array([0.0] + edges + [1.0])
    x, w = np.polynomial.legendre.leggauss(order)
    a, b = edges[:-1], edges[1:]
    X = (a[:, None] + b[:, None]) / 2 + (b - a)[:, None] / 2 * x[None, :]
    W = (b - a)[:, None] / 2 * w[None, :]
    return X.ravel(), W.ravel()


@pytest.fixture(scope="module")
def grid2d():
    X, W = _nodes()
    U, V = np.meshgrid(X, X, indexing="ij")
    return U, V, np.outer(W, W)


# --------------------------------------------------------------------------

def test_ndtri_matches_scipy():
    ps = np.concatenate([np.geomspace(1e-300, 0.5, 400), np.linspace(0.01, 0.5, 200)])
    for p in ps:
        x = oracle.ndtri_lower(p)
        ref = special.ndtri(p)
        assert abs(x - ref) <= 4e-15 * max(1.0, abs(ref)), (p, x, ref)


def test_ranks_match_bruteforce_with_ties():
    g = np.random.default_rng(0)
    for trial in range(40):
        m = int(g.integers(2, 60))
        x = g.integers(0, 6, m).astype(np.float64) * 0.5  # many ties
        if trial % 3 == 0:
            x[g.integers(0, m)] = -0.0
            x[g.integers(0, m)] = 0.0
        off = [0, m]
        r = oracle.ranks(x, off)
        brute = np.array([1 + sum((x[j] < x[i]) or (x[j] == x[i] and j < i) for j in range(m))
                          for i in range(m)])
        assert np.array_equal(r, brute)
        assert sorted(r) == list(range(1, m + 1))


def test_ranks_are_per_subset_and_float32_exact():
    g = np.random.default_rng(1)
    x = g.random(1000).astype(np.float32)
    off = np.array([0, 100, 101 + 1, 500, 1000])
    r = oracle.ranks(x, off)
    for k in range(4):
        seg = x[off[k]:off[k + 1]].astype(np.float64)
        want = np.empty(len(seg), np.int32)
        want[np.argsort(seg, kind="stable")] = np.arange(1, len(seg) + 1)
        assert np.array_equal(r[off[k]:off[k + 1]], want)


def test_ranks_reject_nan():
    with pytest.raises(ValueError):
        oracle.ranks(np.array([0.1, np.nan, 0.3]), [0, 3])


@pytest.mark.parametrize("fam,theta", [(0, 0.3), (0, -0.8), (1, 5.0), (1, -3.0), (1, 0.0004),
                                       (2, 1.0), (2, 2.0), (2, 5.0)])
def test_density_integrates_to_one(fam, theta, grid2d):
    U, V, WW = grid2d
    c = oracle.density(fam, theta, U.ravel(), V.ravel()).reshape(U.shape)
    assert abs((c * WW).sum() - 1.0) < 5e-8


def _frank_C(t, u, v):  # Eq. 10
    return -1.0 / t * np.log(1.0 + (np.exp(-t * u) - 1.0) * (np.exp(-t * v) - 1.0) / (np.exp(-t) - 1.0))


def _gumbel_C(t, u, v):  # Eq. 11
    return np.exp(-(((-np.log(u)) ** t + (-np.log(v)) ** t) ** (1.0 / t)))


@pytest.mark.parametrize("fam,C,theta", [(1, _frank_C, 5.0), (1, _frank_C, -4.0), (1, _frank_C, 0.7),
                                         (2, _gumbel_C, 1.0), (2, _gumbel_C, 2.0), (2, _gumbel_C, 4.0)])
def test_density_is_mixed_derivative_of_paper_copula(fam, C, theta):
    """Eq. 5: c = d^2 C / du dv, with C written from Eq. 10 / Eq. 11."""
    g = np.random.default_rng(2)
    h = 1e-4
    for _ in range(20):
        u, v = g.uniform(0.05, 0.95, 2)
        fd = (C(theta, u + h, v + h) - C(theta, u + h, v - h) - C(theta, u - h, v + h) +
              C(theta, u - h, v - h)) / (4 * h * h)
        c = oracle.density(fam, theta, [u], [v])[0]
        assert abs(c - fd) <= 2e-6 * max(1.0, c), (u, v, c, fd)


def test_gaussian_density_matches_bivariate_normal():
    g = np.random.default_rng(3)
    for rho in (0.3, 0.5, -0.9):
        mvn = stats.multivariate_normal(mean=[0, 0], cov=[[1, rho], [rho, 1]])
        for _ in range(20):
            u, v = g.uniform(1e-6, 1 - 1e-6, 2)
            x, y = special.ndtri(u), special.ndtri(v)
            ref = mvn.pdf([x, y]) / (stats.norm.pdf(x) * stats.norm.pdf(y))
            c = oracle.density(0, rho, [u], [v])[0]
            assert abs(c - ref) <= 1e-10 * ref


def _read_triples():
    rows = []
    with open(os.path.join(GOLDEN, "paper_dependence_triples.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, th, rs, tau = line.split()
                rows.append((cs.FAMILY_NAMES and {"gaussian": 0, "frank": 1, "gumbel": 2}[name],
                             float(th), float(rs), float(tau)))
    return rows


def test_spearman_and_kendall_match_paper(grid2d):
    """Section 2.5 prints Spearman's rho and Kendall's tau for each simulation
    parameter; recover them from the oracle's densities by quadrature."""
    U, V, WW = grid2d
    for fam, th, rs_paper, tau_paper in _read_triples():
        c = oracle.density(fam, th, U.ravel(), V.ravel()).reshape(U.shape)
        rho_s = 12.0 * (U * V * c * WW).sum() - 3.0
        assert round(rho_s, 2) == rs_paper, (fam, rho_s)
        if fam == 1:
            C = _frank_C(th, U, V)
        elif fam == 2:
            C = _gumbel_C(th, U, V)
        else:
            continue  # no closed-form C for Eq. 8; its tau is pinned below
        tau = 4.0 * (C * c * WW).sum() - 1.0
        assert round(tau, 2) == tau_paper, (fam, tau)
    # Gaussian: Spearman's rho has the closed form (6/pi) asin(rho/2)
    c = oracle.density(0, 0.3, U.ravel(), V.ravel()).reshape(U.shape)
    assert abs(12.0 * (U * V * c * WW).sum() - 3.0 - 6 / math.pi * math.asin(0.15)) < 1e-9
    assert round(2 / math.pi * math.asin(0.3), 2) == 0.19


FD_CASES = [(0, 0.5), (0, -0.7), (0, 0.95), (1, 5.0), (1, -3.0), (1, 0.02), (1, 18.0), (1, -0.0006),
            (1, 0.0009), (2, 1.3), (2, 2.0), (2, 7.0)]


@pytest.mark.parametrize("fam,theta", FD_CASES)
def test_score_hessian_and_mixed_partials_by_finite_differences(fam, theta):
    g = np.random.default_rng(4)
    pts = [(0.3, 0.6), (0.02, 0.97), (0.9, 0.85), (0.5, 0.5), (0.999, 0.998), (0.001, 0.003)]
    pts += [tuple(g.uniform(0.01, 0.99, 2)) for _ in range(10)]
    for u, v in pts:
        t = oracle.terms_at(fam, theta, u, v)
        h = 1e-5 * max(1.0, abs(theta))
        if fam == 1 and abs(theta) < 1e-3:
            h = 1e-4  # stay on the series side where the series is used
        tp, tm = oracle.terms_at(fam, theta + h, u, v), oracle.terms_at(fam, theta - h, u, v)
        fd_g = (tp[0] - tm[0]) / (2 * h)
        fd_h = (tp[1] - tm[1]) / (2 * h)
        hu = 1e-6 * min(u, 1 - u, v, 1 - v) / 0.001 if min(u, 1 - u, v, 1 - v) < 0.01 else 1e-6
        fd_tu = (oracle.terms_at(fam, theta, u + hu, v)[1] - oracle.terms_at(fam, theta, u - hu, v)[1]) / (2 * hu)
        fd_tv = (oracle.terms_at(fam, theta, u, v + hu)[1] - oracle.terms_at(fam, theta, u, v - hu)[1]) / (2 * hu)
        for got, fd in ((t[1], fd_g), (t[2], fd_h), (t[3], fd_tu), (t[4], fd_tv)):
            assert abs(got - fd) <= 2e-5 * max(1.0, abs(got)), (fam, theta, u, v, t, fd_g, fd_h, fd_tu, fd_tv)


def test_frank_series_matches_closed_form_at_switch():
    for u, v in [(0.3, 0.6), (0.05, 0.9), (0.7, 0.71)]:
        for t in (9.99e-4, -9.99e-4):
            s = oracle.terms_at(1, t, u, v)          # series side
            d = oracle.terms_at(1, t * 1.0021, u, v)  # closed-form side, just across
            assert np.allclose(s[1:], d[1:], rtol=0, atol=2e-5)
    # independence: c == 1 at theta == 0 exactly
    assert abs(oracle.terms_at(1, 0.0, 0.3, 0.8)[0]) == 0.0


def test_frank_negative_theta_is_v_flip():
    for u, v, t in [(0.3, 0.6, 3.0), (0.05, 0.97, 7.5), (0.8, 0.1, 0.5)]:
        a = oracle.terms_at(1, -t, u, v)
        b = oracle.terms_at(1, t, u, 1 - v)
        assert abs(a[0] - b[0]) < 1e-12 and abs(a[1] + b[1]) < 1e-10 and abs(a[2] - b[2]) < 1e-10


def _subset_ranks(d, k=0):
    lo, hi = d.offsets[k], d.offsets[k + 1]
    m = hi - lo
    return oracle.ranks(d.u[lo:hi], [0, m]), oracle.ranks(d.v[lo:hi], [0, m])


@pytest.mark.parametrize("m,rho", [(1000, 0.5), (200, -0.3), (50, 0.9), (5000, 0.05)])
def test_gaussian_fit_is_root_of_cubic(m, rho):
    """For the Gaussian copula the score vanishes at a real root of
    m r^3 - B r^2 + (A - m) r - B with A = sum(x^2 + y^2), B = sum(x y),
    x = Phi^{-1}(u), y = Phi^{-1}(v); the MPL is the root with the largest l."""
    d = cs.make_dataset(0, rho, m, 1, np.float64, seed=11 + m)
    ru, rv = _subset_ranks(d)
    x = special.ndtri(ru / (m + 1.0))
    y = special.ndtri(rv / (m + 1.0))
    A, B = float(np.sum(x * x + y * y)), float(np.sum(x * y))
    roots = [r.real for r in np.roots([m, -B, A - m, -B]) if abs(r.imag) < 1e-12 and abs(r.real) < 1]

    def ll(r):
        return -0.5 * m * math.log(1 - r * r) - (r * r * A - 2 * r * B) / (2 * (1 - r * r))

    best = max(roots, key=ll)
    th, var, info, st, it = oracle.fit_ranks(0, ru, rv)
    assert st == oracle.OK
    assert abs(th - best) <= 1e-11 * max(1.0, abs(best)), (th, best)


@pytest.mark.parametrize("fam,theta", [(0, 0.4), (1, 4.0), (1, -2.0), (2, 1.7), (2, 3.0)])
def test_fit_matches_bruteforce_on_tiny_subsets(fam, theta):
    g = np.random.default_rng(5)
    for trial in range(6):
        m = int(g.integers(8, 40))
        d = cs.make_dataset(fam, theta, m, 1, np.float64, seed=100 + trial * 7 + fam)
        ru, rv = _subset_ranks(d)
        th, var, info, st, it = oracle.fit_ranks(fam, ru, rv)
        lo, hi = {0: (-0.999, 0.999), 1: (-50, 50), 2: (1.0, 50.0)}[fam]
        grid = np.linspace(lo, hi, 4001)
        ls = np.array([oracle.loglik(fam, t, ru, rv)[0] for t in grid])
        j = int(np.argmax(ls))
        a, b = grid[max(j - 1, 0)], grid[min(j + 1, len(grid) - 1)]
        for _ in range(100):  # golden section on the brute-force cell
            c1, c2 = b - 0.618 * (b - a), a + 0.618 * (b - a)
            if oracle.loglik(fam, c1, ru, rv)[0] > oracle.loglik(fam, c2, ru, rv)[0]:
                b = c2
            else:
                a = c1
        tb = 0.5 * (a + b)
        if st in (oracle.BOUNDARY, oracle.CAPPED):
            assert abs(th - tb) < 1e-3
        else:
            assert abs(th - tb) <= 1e-6 * max(1.0, abs(tb)), (fam, m, th, tb)
            assert oracle.loglik(fam, th, ru, rv)[0] >= ls.max() - 1e-9


@pytest.mark.parametrize("fam,theta,m", [(0, 0.5, 3000), (1, 5.0, 3000), (1, -1.5, 800),
                                         (2, 2.0, 3000), (2, 1.1, 500)])
def test_score_vanishes_at_optimum(fam, theta, m):
    d = cs.make_dataset(fam, theta, m, 1, np.float32, seed=200 + m + fam)
    ru, rv = _subset_ranks(d)
    th, var, info, st, it = oracle.fit_ranks(fam, ru, rv)
    if st == oracle.BOUNDARY:
        assert fam == 2 and th == 1.0 and oracle.loglik(fam, 1.0, ru, rv)[1] <= 0
        return
    l, gsum, h = oracle.loglik(fam, th, ru, rv)
    assert h < 0
    # score scale: sum |l_t| over the subset
    scale = sum(abs(oracle.point(fam, th, int(a), int(b), m)[1]) for a, b in zip(ru[:200], rv[:200])) * m / 200
    assert abs(gsum) <= 1e-10 * scale, (gsum, scale)


@pytest.mark.parametrize("fam,theta", [(0, 0.5), (1, 5.0), (2, 2.0), (2, 5.0), (1, -4.0)])
def test_large_n_recovers_generating_parameter(fam, theta):
    n = 60_000
    d = cs.make_dataset(fam, theta, n, 1, np.float64, seed=300 + fam)
    r = oracle.fit(fam, d.u, d.v, d.offsets)
    sd = math.sqrt(r["var"][0])
    assert r["status"][0] == oracle.OK
    assert abs(r["theta"][0] - theta) <= 4.5 * sd, (r["theta"][0], theta, sd)


def test_variance_direct_equals_suffix_scan():
    for fam, theta in [(0, 0.5), (1, 5.0), (2, 2.0), (1, -2.0)]:
        d = cs.make_dataset(fam, theta, 700, 1, np.float32, seed=400 + fam)
        ru, rv = _subset_ranks(d)
        th = oracle.fit_ranks(fam, ru, rv)[0]
        a = oracle.var_at(fam, th, ru, rv, True)
        b = oracle.var_at(fam, th, ru, rv, False)
        assert abs(a - b) <= 1e-12 * abs(a)


def _plug_in_sandwich(ru, rv, lt, ltt, ltu, ltv):
    """Var(theta_hat) = sigma^2 / m of one subset by the plug-in sandwich of
    Genest, Ghoudi & Rivest (1995) written as dense O(m^2) indicator
    matrices: W1_i = (1/m) sum_j [U_i <= U_j] l_tu(j), W2 likewise in V,
    xi = l_t + W1 + W2, nu^2 = mean((xi - mean xi)^2), beta = -mean l_tt."""
    m = ru.shape[0]
    Iu = (ru[:, None] <= ru[None, :]).astype(np.float64)
    Iv = (rv[:, None] <= rv[None, :]).astype(np.float64)
    xi = lt + (Iu @ ltu) / m + (Iv @ ltv) / m
    nu2 = np.mean((xi - xi.mean()) ** 2)
    beta = -np.mean(ltt)
    return nu2 / beta ** 2 / m


@pytest.mark.parametrize("fam,theta,m", [(1, 5.0, 500), (1, -2.5, 311), (1, 0.6, 120), (2, 2.0, 500),
                                         (2, 4.5, 257), (2, 1.3, 90), (0, 0.5, 400), (0, -0.7, 150)])
def test_variance_equals_brute_force_plug_in_sandwich(fam, theta, m):
    """The oracle's variance (both its O(m^2) loop and its rank-order suffix
    form) against a separately written dense-matrix plug-in sandwich on the
    oracle's per-point terms, to rounding: a slip in the W terms (direction,
    normaliser, a dropped W, the wrong margin) moves the variance by far more
    than 1e-12."""
    d = cs.make_dataset(fam, theta, m, 1, np.float64, seed=410 + m)
    ru, rv = _subset_ranks(d)
    th = oracle.fit_ranks(fam, ru, rv)[0]
    P = np.array([oracle.point(fam, th, int(a), int(b), m) for a, b in zip(ru, rv)])
    want = _plug_in_sandwich(ru, rv, P[:, 1], P[:, 2], P[:, 3], P[:, 4])
    for direct in (True, False):
        got = oracle.var_at(fam, th, ru, rv, direct)
        assert abs(got - want) <= 1e-12 * abs(want), (fam, theta, m, direct, got, want)


@pytest.mark.parametrize("fam,theta", [(1, 4.0), (2, 2.5), (0, 0.4)])
def test_variance_with_finite_difference_mixed_partials(fam, theta):
    """The same sandwich with l_tu and l_tv taken by central differences of
    the oracle's score in u and v (not its analytic mixed partials) agrees
    to the differencing error."""
    m = 300
    d = cs.make_dataset(fam, theta, m, 1, np.float64, seed=470 + fam)
    ru, rv = _subset_ranks(d)
    th = oracle.fit_ranks(fam, ru, rv)[0]
    P = np.array([oracle.point(fam, th, int(a), int(b), m) for a, b in zip(ru, rv)])
    u, v = ru / (m + 1.0), rv / (m + 1.0)
    h = 1e-6
    ltu = np.array([(oracle.terms_at(fam, th, a + h, b)[1] - oracle.terms_at(fam, th, a - h, b)[1]) / (2 * h)
                    for a, b in zip(u, v)])
    ltv = np.array([(oracle.terms_at(fam, th, a, b + h)[1] - oracle.terms_at(fam, th, a, b - h)[1]) / (2 * h)
                    for a, b in zip(u, v)])
    want = _plug_in_sandwich(ru, rv, P[:, 1], P[:, 2], ltu, ltv)
    got = oracle.var_at(fam, th, ru, rv, False)
    assert abs(got - want) <= 1e-6 * abs(want), (fam, got, want)


def test_gaussian_variance_closed_form():
    """For the Gaussian copula the MPL estimator's asymptotic variance is
    (1 - rho^2)^2 (Genest, Ghoudi & Rivest 1995; Klaassen & Wellner 1997)."""
    rho, n = 0.5, 40_000
    d = cs.make_dataset(0, rho, n, 1, np.float64, seed=500)
    r = oracle.fit(0, d.u, d.v, d.offsets)
    assert abs(n * r["var"][0] / (1 - rho * rho) ** 2 - 1.0) < 0.04


def test_variance_matches_monte_carlo():
    fam, theta, m, R = 1, 5.0, 400, 150
    ths, vs = [], []
    for rep in range(R):
        d = cs.make_dataset(fam, theta, m, 1, np.float64, seed=10_000 + rep)
        ru, rv = _subset_ranks(d)
        th, var, info, st, it = oracle.fit_ranks(fam, ru, rv)
        ths.append(th)
        vs.append(var)
    ratio = np.var(ths) / np.mean(vs)
    assert 0.72 < ratio < 1.38, ratio


def test_combine_hand_arithmetic():
    th = np.array([1.0, 2.0, 4.0])
    var = np.array([1.0, 0.5, 0.25])
    info = np.array([3.0, 1.0, 0.0])
    st = np.zeros(3, np.int32)
    # Eq. 15: w = 1/var = (1, 2, 4): (1 + 4 + 16) / 7 = 3
    assert oracle.combine(th, var, info, st, oracle.W_INVVAR) == 3.0
    assert oracle.combine(th, var, info, st, oracle.W_EQUAL) == pytest.approx(7.0 / 3.0, abs=1e-15)
    # Fisher weights 3, 1, (0 -> dropped): (3 + 2) / 4
    assert oracle.combine(th, var, info, st, oracle.W_FISHER) == 1.25
    st[2] = oracle.DEGENERATE
    assert oracle.combine(th, var, info, st, oracle.W_INVVAR) == pytest.approx(5.0 / 3.0, abs=1e-15)
    st[2] = oracle.CAPPED
    assert oracle.combine(th, var, info, st, oracle.W_INVVAR) == pytest.approx(5.0 / 3.0, abs=1e-15)
    st[2] = oracle.BOUNDARY
    assert oracle.combine(th, var, info, st, oracle.W_INVVAR) == 3.0


def test_tiny_subsets_hit_the_caps():
    # two concordant points: the likelihood rises without bound in theta
    for fam, cap in ((0, 1 - 1e-9), (1, 50.0), (2, 50.0)):
        th, var, info, st, it = oracle.fit_ranks(fam, np.array([1, 2]), np.array([1, 2]))
        assert st == oracle.CAPPED and th == cap
    th, var, info, st, it = oracle.fit_ranks(2, np.array([1, 2]), np.array([2, 1]))
    assert st == oracle.BOUNDARY and th == 1.0


def test_fit_combines_subsets_in_order():
    d = cs.make_dataset(1, 5.0, 3000, 3, np.float32, seed=600)
    r = oracle.fit(1, d.u, d.v, d.offsets, nthreads=3)
    w = 1.0 / r["var"]
    assert abs(r["combined"] - float(np.sum(w * r["theta"]) / np.sum(w))) < 1e-14
    r1 = oracle.fit(1, d.u, d.v, d.offsets, nthreads=1)
    assert np.array_equal(r["theta"], r1["theta"]) and np.array_equal(r["var"], r1["var"])


def test_fit_rejects_bad_partitions():
    u = np.linspace(0.1, 0.9, 10)
    with pytest.raises(ValueError):
        oracle.fit(1, u, u, [0, 1, 10])  # subset of size 1
    with pytest.raises(ValueError):
        oracle.fit(1, u, u, [0, 5, 9])  # does not cover n
