"""Host-side arithmetic of bench.py (no GPU): the per-pass metric's pass
counts, the algorithmic work counts behind the roofline, and the theta-error
summaries against the oracle."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_gaussian_counts_one_pass_others_their_newton_passes():
    p = bench.passes_per_subset([0, 1, 2, 0], [0, 3, 4, 7])
    assert p.tolist() == [1.0, 3.0, 4.0, 1.0]


def test_work_counts_by_hand():
    m = np.array([1000, 2000, 500])
    fams = np.array([0, 1, 2])
    it = np.array([0, 3, 5])
    pp, mufu, hbm = bench.work_counts(m, fams, it)
    assert pp == 1000 * 1 + 2000 * 3 + 500 * 5
    # Gaussian: 2 quantiles per pair once; Frank: 4 per pass, (3 + 2 variance) passes;
    # Gumbel: 7 per pass, (5 + 2) passes, plus 4 once
    assert mufu == 1000 * 2 + 2000 * 4 * 5 + 500 * (7 * 7 + 4)
    assert hbm == 3500 * 8 + 3 * 20


def test_theta_errors_relative_away_from_zero_absolute_near_it():
    o = np.array([2.0, -1.0, 0.01, 0.5, 3.0])
    g = np.array([2.0 + 2e-6, -1.0 - 1e-6, 0.01 + 3e-8, 0.5, 3.0])
    st_o = np.array([0, 0, 0, 3, 1])
    st_g = np.array([0, 0, 0, 0, 1])
    e = bench.theta_errors(g, st_g, o, st_o)
    assert e["compared"] == 4 and e["status_mismatch"] == 1
    assert e["max_rel"] == pytest.approx(1e-6, rel=1e-6)
    assert e["near_zero"] == 1 and e["max_abs_near_zero"] == pytest.approx(3e-8, rel=1e-6)
    c = bench.combined_errors([1.0 + 1e-7, 0.02], [1.0, 0.0200001])
    assert c["compared"] == 2 and c["max_rel"] == pytest.approx(2e-6, rel=1e-3)


def test_replica_throughput_counts_every_rank():
    assert bench.replica_throughput(4, 1e6, 10, 2.0) == 2e7
