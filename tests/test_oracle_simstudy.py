"""Pins of the oracle's simulation-study summaries (Section 2.5-2.6, CPU only).

Eq. 17-18 average the per-simulation combined and full-data estimates; the
estimated bias and MSE compare them; Eq. 19-20 are relative L1 / L2 distances
between the copula densities at the two averaged parameters, integrated over
[delta, 1-delta]^2.  Pinned against: the unit mass of every copula density,
the closed form int int c^2 = 1 / (1 - rho^2) of the Gaussian copula, a
first-order expansion in the parameter built from the oracle's separately
pinned score l_theta, the finiteness of the Frank norms, the logarithmic
growth of the Gumbel squared norms near (1, 1), and hand arithmetic.
"""
import math

import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("fam,theta,delta", [(0, 0.3, 0.0), (0, -0.7, 0.0), (1, 5.0, 0.0), (1, -12.0, 0.0),
                                             (2, 1.5, 0.0), (2, 5.0, 0.0)])
def test_every_density_has_unit_mass(fam, theta, delta):
    s = oracle.density_integrals(fam, theta, theta, delta)
    assert s[0] == 0.0 and s[2] == 0.0
    assert abs(s[1] - 1.0) < (1e-9 if fam != 2 else 1e-5), s[1]


@pytest.mark.parametrize("rho", [0.3, -0.5])
def test_gaussian_squared_norm_closed_form(rho):
    """int int c^2 = 2 pi / sqrt(det M) / (2 pi (1 - rho^2)) with
    M = 2 Sigma^-1 - I, whose determinant is 1.  (Moderate dependence: the
    product rule does not follow the diagonal ridge of strong dependence.)"""
    s = oracle.density_integrals(0, rho, rho, 0.0)
    assert abs(s[3] - 1.0 / (1.0 - rho * rho)) < 1e-9 * s[3], (s[3], 1.0 / (1.0 - rho * rho))


def test_gumbel_underflow_is_an_error():
    with pytest.raises(ValueError):
        oracle.density_integrals(2, 50.0, 50.0, 1e-9)


def _first_order(fam, theta, dtheta, delta):
    """|dtheta| int int |c l_theta| and dtheta^2 int int (c l_theta)^2 on a
    plain Gauss-Legendre grid, from the oracle's pinned per-point terms."""
    x, w = np.polynomial.legendre.leggauss(200)
    a, b = delta if delta > 0 else 1e-6, 1 - (delta if delta > 0 else 1e-6)
    X = 0.5 * (a + b) + 0.5 * (b - a) * x
    W = 0.5 * (b - a) * w
    l1 = l2 = 0.0
    for i, u in enumerate(X):
        for j, v in enumerate(X):
            t = oracle.terms_at(fam, theta, u, v)
            d = math.exp(t[0]) * t[1]
            l1 += W[i] * W[j] * abs(d)
            l2 += W[i] * W[j] * d * d
    return abs(dtheta) * l1, dtheta * dtheta * l2


def test_small_parameter_change_matches_first_order_expansion():
    """Frank (bounded density): the distance integrals for theta + dtheta
    equal the first-order terms built from the score l_theta."""
    th, dth = 5.0, 1e-4
    s = oracle.density_integrals(1, th, th + dth, 0.0)
    e1, e2 = _first_order(1, th, dth, 0.0)
    assert abs(s[0] - e1) < 2e-3 * e1, (s[0], e1)
    assert abs(s[2] - e2) < 4e-3 * e2, (s[2], e2)


def test_frank_norms_are_finite():
    a = oracle.density_integrals(1, 8.0, 8.0, 0.0)[3]
    b = oracle.density_integrals(1, 8.0, 8.0, 1e-9)[3]
    assert abs(a - b) < 1e-7 * a


def test_gumbel_squared_norm_grows_like_log_inverse_delta():
    """The Gumbel density is of order 1/|(1-u, 1-v)| near (1, 1), so
    int int c^2 over [delta, 1-delta]^2 grows linearly in log(1/delta); the
    relative L2 distance (a ratio of two such integrals) still settles."""
    s = [oracle.density_integrals(2, 5.0, 5.01, d) for d in (1e-3, 1e-6, 1e-9)]
    g1, g2 = s[1][3] - s[0][3], s[2][3] - s[1][3]
    assert g1 > 1.0 and abs(g2 - g1) < 0.05 * g1, (g1, g2)
    d2 = [math.sqrt(x[2] / x[3]) for x in s]
    assert abs(d2[2] - d2[1]) < abs(d2[1] - d2[0])


@pytest.mark.parametrize("fam,a,b,delta", [(0, 0.3, 0.35, 0.0), (1, 5.0, 4.0, 0.0), (2, 5.0, 6.0, 1e-6)])
def test_norms_of_the_first_density_do_not_see_the_second(fam, a, b, delta):
    """out[1] and out[3] are norms of c(.; theta_a) alone, and the distance
    integrals are symmetric in the two parameters."""
    s_ab = oracle.density_integrals(fam, a, b, delta)
    s_aa = oracle.density_integrals(fam, a, a, delta)
    s_ba = oracle.density_integrals(fam, b, a, delta)
    assert s_ab[1] == s_aa[1] and s_ab[3] == s_aa[3]
    assert abs(s_ab[0] - s_ba[0]) < 1e-14 * s_ab[0] and abs(s_ab[2] - s_ba[2]) < 1e-14 * s_ab[2]


def test_relative_distances_are_the_ratios():
    d1, d2 = oracle.relative_distances(1, 5.0, 5.2, 0.0)
    s = oracle.density_integrals(1, 5.0, 5.2, 0.0)
    assert d1 == s[0] / s[1] and d2 == math.sqrt(s[2] / s[3])
    assert oracle.relative_distances(0, 0.3, 0.3) == (0.0, 0.0)


def test_simulation_summary_by_hand():
    comb = [2.0, 2.2, 1.9, 2.1]
    full = [2.0, 2.0, 2.0, 2.0]
    r = oracle.simulation_summary(comb, full)
    assert abs(r["theta_combined_sim"] - 2.05) < 1e-15   # Eq. 17
    assert r["theta_full_sim"] == 2.0                    # Eq. 18
    assert abs(r["bias"] - 0.05) < 1e-15
    assert abs(r["mse"] - (0 + 0.04 + 0.01 + 0.01) / 4) < 1e-15
