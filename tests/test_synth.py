"""The seeded input generators: each sampler reproduces its copula's Kendall tau,
and the partitions follow Eq. 14 (contiguous, covering, sizes as specified)."""
import numpy as np
import pytest
from scipy import stats

import copula_synth as cs


@pytest.mark.parametrize("fam,theta", [(0, 0.5), (1, 5.0), (1, -3.0), (2, 2.0), (2, 5.0)])
def test_sampler_kendall_tau(fam, theta):
    u, v = cs.sample(fam, theta, 20_000, cs.rng(7 + fam))
    assert np.all((u > 0) & (u < 1) & (v > 0) & (v < 1))
    tau = stats.kendalltau(u, v)[0]
    assert abs(tau - cs.tau_of(fam, theta)) < 0.015, (tau, cs.tau_of(fam, theta))


def test_tau_maps():
    # Section 2.5 prints tau = 0.46 for Frank theta = 5 and 0.80 for Gumbel theta = 5
    assert round(cs.tau_of(1, 5.0), 2) == 0.46
    assert round(cs.tau_of(2, 5.0), 2) == 0.80
    for fam in (0, 1, 2):
        for tau in (0.1, 0.46, 0.8):
            assert abs(cs.tau_of(fam, cs.theta_of_tau(fam, tau)) - tau) < 1e-10
    assert abs(cs.theta_of_tau(1, 0.1) - 0.9073) < 1e-3
    assert abs(cs.theta_of_tau(1, 0.8) - 18.19) < 1e-2


def test_partitions():
    off = cs.equal_offsets(10_007, 10)
    assert off[0] == 0 and off[-1] == 10_007 and np.all(np.diff(off) >= 1000)
    off = cs.lognormal_offsets(1_000_000, 1000, 1.0, cs.rng(3))
    sz = np.diff(off)
    assert off[-1] == 1_000_000 and sz.min() >= 2 and len(sz) == 1000
    assert 5 < sz.max() / np.median(sz) < 100


def test_seeded_reproducible():
    a = cs.make_dataset(1, 5.0, 1000, 2, seed=9)
    b = cs.make_dataset(1, 5.0, 1000, 2, seed=9)
    assert np.array_equal(a.u, b.u) and np.array_equal(a.v, b.v)
