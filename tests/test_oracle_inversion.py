"""Pins of the oracle's rank-correlation inversion estimators (CPU only).

Section 2.3 lists the inversion of Kendall's tau and of Spearman's rho among
the estimators the paper does not use, and Section 2.5 prints the population
tau and rho of each generating copula.  The oracle computes the subset
statistics from the ranks, the population values from their textbook forms
(Gaussian arcsine laws, Frank's Debye-function forms, Gumbel's 1 - 1/theta and
a quadrature of its copula) and inverts them.  These tests pin that against
things other than itself: scipy's sample statistics, the values the paper
prints, a quadrature of the oracle's (separately pinned) densities and
copulas, round trips, the edges of the parameter domains, and a large sample.
"""
import math
import os

import numpy as np
import pytest

import copula_synth as cs
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _ranks_of(x):
    r = np.empty(len(x), dtype=np.int32)
    r[np.argsort(x, kind="stable")] = np.arange(1, len(x) + 1)
    return r


def _graded_grid(nsub=40, order=10):
    edges = (list(np.geomspace(1e-12, 0.02, 20)) + list(np.linspace(0.02, 0.98, nsub)[1:-1]) +
             list(1 - np.geomspace(0.02, 1e-12, 20)))
    edges = np.array([0.0] + edges + [1.0])
    x, w = np.polynomial.legendre.leggauss(order)
    a, b = edges[:-1], edges[1:]
    X = ((a[:, None] + b[:, None]) / 2 + (b - a)[:, None] / 2 * x[None, :]).ravel()
    W = ((b - a)[:, None] / 2 * w[None, :]).ravel()
    U, V = np.meshgrid(X, X, indexing="ij")
    return U, V, np.outer(W, W)


@pytest.fixture(scope="module")
def grid2d():
    return _graded_grid()


def test_subset_statistics_match_scipy():
    stats = pytest.importorskip("scipy.stats")
    g = np.random.default_rng(7)
    for m in (2, 3, 17, 500, 2001):
        x = g.standard_normal(m)
        y = 0.6 * x + 0.8 * g.standard_normal(m)
        ru, rv = _ranks_of(x), _ranks_of(y)
        assert abs(oracle.kendall_tau(ru, rv) - stats.kendalltau(x, y)[0]) < 1e-12, m
        assert abs(oracle.spearman_rho(ru, rv) - stats.spearmanr(x, y)[0]) < 1e-12, m
    r = np.arange(1, 101, dtype=np.int32)
    assert oracle.kendall_tau(r, r) == 1.0 and oracle.kendall_tau(r, r[::-1].copy()) == -1.0
    assert oracle.spearman_rho(r, r) == 1.0 and oracle.spearman_rho(r, r[::-1].copy()) == -1.0


def test_merge_count_tau_equals_every_pair_count():
    """The oracle's O(m log m) Kendall's tau (inversions of the v-ranks in
    u-rank order, by merge sort) equals its every-pair definition bit for bit,
    on random, sorted, reversed and strongly dependent subsets of odd and
    power-of-two sizes; and scipy's tau on a larger sample."""
    g = np.random.default_rng(11)
    for m in (2, 3, 7, 64, 257, 1024, 3001):
        for kind in ("random", "sorted", "reversed", "dependent"):
            x = g.standard_normal(m)
            y = {"random": g.standard_normal(m), "sorted": x.copy(), "reversed": -x,
                 "dependent": 0.9 * x + 0.3 * g.standard_normal(m)}[kind]
            ru, rv = _ranks_of(x), _ranks_of(y)
            assert oracle.kendall_tau_merge(ru, rv) == oracle.kendall_tau(ru, rv), (m, kind)
    stats = pytest.importorskip("scipy.stats")
    x = g.standard_normal(200_000)
    y = 0.5 * x + g.standard_normal(200_000)
    assert abs(oracle.kendall_tau_merge(_ranks_of(x), _ranks_of(y)) - stats.kendalltau(x, y)[0]) < 1e-12


def test_population_values_match_the_paper():
    """Section 2.5 prints rho_S and tau (two decimals) beside each parameter."""
    names = {"gaussian": 0, "frank": 1, "gumbel": 2}
    with open(os.path.join(GOLDEN, "paper_dependence_triples.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    for name, th, rs, tau in rows:
        fam = names[name]
        assert round(oracle.rho_s_of_theta(fam, float(th)), 2) == float(rs), name
        assert round(oracle.tau_of_theta(fam, float(th)), 2) == float(tau), name


@pytest.mark.parametrize("fam,theta", [(1, -3.0), (1, 0.5), (1, 2.0), (1, 8.0), (1, 20.0),
                                       (2, 1.2), (2, 2.0), (2, 5.0)])
def test_population_values_match_density_quadrature(fam, theta, grid2d):
    """tau = 4 E[C(U,V)] - 1 and rho_S = 12 E[U V] - 3 under the copula,
    integrated against the oracle's density (its own pins: unit mass, mixed
    second difference of Eq. 10 / Eq. 11)."""
    U, V, WW = grid2d
    c = oracle.density(fam, theta, U.ravel(), V.ravel()).reshape(U.shape)
    C = np.vectorize(lambda a, b: oracle.cdf(fam, theta, a, b))(U, V)
    tau_q = 4.0 * (C * c * WW).sum() - 1.0
    rho_q = 12.0 * (U * V * c * WW).sum() - 3.0
    tol = 1e-7 if fam == 1 else 2e-4  # Gumbel's density is unbounded at (1, 1)
    assert abs(oracle.tau_of_theta(fam, theta) - tau_q) < tol, (tau_q, oracle.tau_of_theta(fam, theta))
    assert abs(oracle.rho_s_of_theta(fam, theta) - rho_q) < tol, (rho_q, oracle.rho_s_of_theta(fam, theta))


@pytest.mark.parametrize("theta", [1.01, 1.2, 2.0, 5.0, 20.0, 50.0])
def test_gumbel_spearman_matches_pickands_form(theta):
    """Gumbel is an extreme-value copula with Pickands dependence function
    A(t) = (t^theta + (1-t)^theta)^(1/theta), and for such copulas
    rho_S = 12 int_0^1 (1 + A(t))^-2 dt - 3: a one-dimensional route, split
    at t = 1/2 where A has its ridge, independent of the oracle's
    two-dimensional integral of C."""
    x, w = np.polynomial.legendre.leggauss(400)
    s = 0.0
    for a, b in ((0.0, 0.5), (0.5, 1.0)):
        t = 0.5 * (b - a) * x + 0.5 * (a + b)
        A = (t ** theta + (1 - t) ** theta) ** (1 / theta)
        s += np.sum(0.5 * (b - a) * w / (1 + A) ** 2)
    assert abs(oracle.rho_s_of_theta(2, theta) - (12 * s - 3)) < 1e-10


@pytest.mark.parametrize("rho", [-0.6, 0.3, 0.8])
def test_gaussian_spearman_matches_density_quadrature(rho, grid2d):
    U, V, WW = grid2d
    c = oracle.density(0, rho, U.ravel(), V.ravel()).reshape(U.shape)
    assert abs(oracle.rho_s_of_theta(0, rho) - (12.0 * (U * V * c * WW).sum() - 3.0)) < 1e-7


def test_gaussian_tau_matches_a_large_sample():
    """The arcsine law for tau against the sample tau of 20,000 Gaussian-copula
    pairs (standard error about 0.004)."""
    d = cs.make_dataset(0, 0.5, 20_000, 1, np.float64, seed=808)
    t = oracle.kendall_tau(_ranks_of(d.u), _ranks_of(d.v))
    assert abs(t - oracle.tau_of_theta(0, 0.5)) < 0.02
    assert abs(oracle.tau_of_theta(0, 0.5) - 1.0 / 3.0) < 1e-15  # (2/pi) asin(1/2)


@pytest.mark.parametrize("fam,thetas", [(0, [-0.9, -0.3, 0.0, 0.45, 0.95]),
                                        (1, [-30.0, -2.0, -1e-3, 1e-5, 0.7, 5.0, 40.0]),
                                        (2, [1.0 + 1e-6, 1.3, 2.0, 5.0, 30.0])])
def test_inversion_round_trips(fam, thetas):
    for th in thetas:
        for fwd, inv in ((oracle.tau_of_theta, oracle.theta_from_tau),
                         (oracle.rho_s_of_theta, oracle.theta_from_rho_s)):
            t, st = inv(fam, fwd(fam, th))
            assert st == oracle.OK, (fam, th, st)
            assert abs(t - th) <= 1e-9 * max(1.0, abs(th)), (fam, th, t)


def test_maps_are_odd_and_increasing():
    for fam, lo, hi in ((0, -0.99, 0.99), (1, -40.0, 40.0)):
        ths = np.linspace(lo, hi, 41)
        for f in (oracle.tau_of_theta, oracle.rho_s_of_theta):
            vals = np.array([f(fam, t) for t in ths])
            assert np.all(np.diff(vals) > 0), fam
            assert np.allclose(vals, -vals[::-1], atol=1e-13), fam
    g = np.array([oracle.rho_s_of_theta(2, t) for t in np.linspace(1.0, 20.0, 20)])
    assert np.all(np.diff(g) > 0) and abs(g[0]) < 1e-9


def test_frank_near_independence():
    """tau ~ theta/9 - theta^3/900 and rho_S ~ theta/6 - theta^3/450 as
    theta -> 0, and the series and the Debye closed forms agree where they
    meet (|theta| = 0.5)."""
    for th in (1e-6, 1e-4, 1e-2):
        assert abs(oracle.tau_of_theta(1, th) - (th / 9.0 - th ** 3 / 900.0)) < 1e-12 * th
        assert abs(oracle.rho_s_of_theta(1, th) - (th / 6.0 - th ** 3 / 450.0)) < 1e-12 * th
    below = float(np.nextafter(0.5, 0.0))  # the last series point; 0.5 takes the closed form
    for f in (oracle.tau_of_theta, oracle.rho_s_of_theta):
        assert abs(f(1, 0.5) - f(1, below)) < 1e-12


def test_inversion_edges():
    assert oracle.theta_from_tau(2, -0.1) == (1.0, oracle.BOUNDARY)
    assert oracle.theta_from_rho_s(2, 0.0) == (1.0, oracle.BOUNDARY)
    assert oracle.theta_from_tau(2, 0.99)[1] == oracle.CAPPED   # theta = 100 > 50
    assert oracle.theta_from_tau(1, 0.95)[1] == oracle.CAPPED   # Frank tau(50) ~ 0.92
    assert oracle.theta_from_tau(1, -0.95)[1] == oracle.CAPPED
    assert oracle.theta_from_tau(0, 1.0)[1] == oracle.CAPPED
    th, st = oracle.theta_from_tau(0, -1.0 / 3.0)
    assert st == oracle.OK and abs(th + 0.5) < 1e-15
    assert oracle.theta_from_tau(1, math.nan)[1] == oracle.DEGENERATE


@pytest.mark.parametrize("fam,theta", [(1, 5.0), (2, 2.0)])
def test_tau_inversion_recovers_the_generating_parameter(fam, theta):
    """On 20,000 generated pairs the tau- and rho-inversion estimates lie
    within five standard errors of theta (standard error of the sample tau
    and rho about 0.005, mapped through the slope of the inverse)."""
    d = cs.make_dataset(fam, theta, 20_000, 1, np.float64, seed=909 + fam)
    ru, rv = _ranks_of(d.u), _ranks_of(d.v)
    for stat, fwd, inv in ((oracle.kendall_tau, oracle.tau_of_theta, oracle.theta_from_tau),
                           (oracle.spearman_rho, oracle.rho_s_of_theta, oracle.theta_from_rho_s)):
        th, st = inv(fam, stat(ru, rv))
        assert st == oracle.OK
        slope = 0.02 / (fwd(fam, theta + 0.01) - fwd(fam, theta - 0.01))
        assert abs(th - theta) < 5 * 0.005 * slope, (stat.__name__, th, theta)
