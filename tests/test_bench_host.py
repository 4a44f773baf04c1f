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
    pp, (ex2, lg2, rcp), hbm = bench.work_counts(m, fams, it)
    assert pp == 1000 * 1 + 2000 * 3 + 500 * 5
    # Gaussian: 2 quantiles (lg2) per pair once; Frank: 3 ex2 + 1 rcp per pass
    # over (3 + 2 variance) passes; Gumbel: 3 ex2 + 2 lg2 + 2 rcp per pass over
    # (5 + 2) passes, plus 4 lg2 once
    assert ex2 == 2000 * 3 * 5 + 500 * 3 * 7
    assert lg2 == 1000 * 2 + 500 * (2 * 7 + 4)
    assert rcp == 2000 * 1 * 5 + 500 * 2 * 7
    assert hbm == 3500 * 8 + 3 * 20


def test_roofline_weights_the_mufu_classes_by_their_rates():
    rates = {"mufu_ex2": 2e12, "mufu_lg2": 1e12, "mufu_rcp": 1e12, "fp32_fma": 3e13, "fp64_fma": 5e11}
    work = (0.0, (2e9, 1e9, 1e9), 8e6)
    r = bench.roofline("x", work, 4.0, rates, {"hbm_gbs": 7000.0}, "measured", None, None, "k", 1)
    # bound time: 2e9/2e12 + 1e9/1e12 + 1e9/1e12 = 3 ms of a 4 ms kernel
    assert r["bound"] == "alu" and abs(r["frac"] - 0.75) < 1e-12
    assert abs(r["achieved"] - 4e9 / 4e-3 / 1e12) < 1e-12 and abs(r["peak"] - 4e9 / 3e-3 / 1e12) < 1e-9


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


def test_fit_phases_split_the_barrier_timestamps():
    """F32C: two sweeps before the Newton passes, a sweep and a step per
    pass, the variance sweeps after; FP64: a third sweep before and three
    barriers around the FP32 start search.  The last span runs to the
    kernel's end."""
    nv = bench.FIT_VARIANCE_BARRIERS
    # F32C with 3 Newton passes: barriers at 1, 2 (tables, Gaussian sums),
    # then 6 for the passes, then nv for the variance
    t = np.cumsum([1.0, 0.5] + [0.2, 0.1] * 3 + [0.3] * nv)
    out = bench.fit_phases(t, float(t[-1]) + 0.25, "f32c")
    assert out["tables"] == pytest.approx(1.0) and out["gaussian_sums"] == pytest.approx(0.5)
    assert out["newton_passes"] == 3 and out["newton"] == pytest.approx(0.9)
    assert len(out["variance_sweeps"]) == nv + 1
    assert out["variance"] == pytest.approx(0.3 * nv + 0.25)
    # FP64: gathered v-table, then 3 barriers of the FP32 start search besides its passes
    t = np.cumsum([1.0, 0.4, 0.5] + [0.7] * 3 + [0.2, 0.1] * 4 + [0.3] * nv)
    out = bench.fit_phases(t, float(t[-1]) + 0.1, "f64")
    assert out["tables"] == pytest.approx(1.4) and out["gaussian_sums"] == pytest.approx(0.5)
    assert out["newton_passes"] == 4
    assert bench.fit_phases(t[:3], 5.0, "f64") is None
