"""The simulation study's summaries on the GPU (Sections 2.5-2.6): the
Eq. 19-20 density integrals against the oracle's quadrature (1e-12 relative;
both use the same stated product rule, so they differ only by rounding), the
Eq. 17-18 means, bias and MSE against the oracle's arithmetic, and a small
study end to end: replicates drawn on the device, GPU fits, GPU summary,
against the oracle's fits and summary of the same replicates."""
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

CASES = [  # family, theta_full, theta_combined, delta
    (0, 0.3, 0.3012, 0.0), (0, 0.5, 0.47, 0.0), (0, -0.4, -0.41, 1e-4),
    (1, 5.0, 5.02, 0.0), (1, -3.0, -2.9, 0.0), (1, 0.5, 0.52, 1e-3),
    (2, 5.0, 5.01, 1e-6), (2, 2.0, 2.05, 1e-3), (2, 1.3, 1.31, 1e-4),
]


@pytest.mark.parametrize("fam,ta,tb,delta", CASES)
def test_density_integrals_match_oracle(fam, ta, tb, delta):
    integ, rel = cg.density_distance(fam, [ta], [tb], delta)
    got = integ.cpu().numpy()[0]
    want = oracle.density_integrals(fam, ta, tb, delta)
    assert np.all(np.abs(got - want) <= 1e-12 * np.abs(want)), (got, want)
    d1, d2 = oracle.relative_distances(fam, ta, tb, delta)
    r = rel.cpu().numpy()[0]
    assert abs(r[0] - d1) <= 1e-12 * d1 and abs(r[1] - d2) <= 1e-12 * d2


def test_density_integrals_batch_of_pairs_equals_single_calls():
    ta = [5.0, 4.0, 6.5, 5.0]
    tb = [5.02, 3.9, 6.4, 5.0]
    integ, _ = cg.density_distance(1, ta, tb, 0.0)
    for k in range(4):
        one, _ = cg.density_distance(1, [ta[k]], [tb[k]], 0.0)
        assert torch.equal(integ[k], one[0])
    assert integ[3, 0].item() == 0.0 and integ[3, 2].item() == 0.0   # equal parameters: zero distance


def test_density_distance_rejects_bad_arguments():
    with pytest.raises(cg.CopulaError):
        cg.density_distance(1, [5.0], [5.0], 0.05)    # delta must stay below 0.02
    with pytest.raises(cg.CopulaError):
        cg.density_distance(3, [5.0], [5.0], 0.0)


@pytest.mark.parametrize("fam,theta,delta", [(0, 0.3, 0.0), (1, 5.0, 0.0), (2, 5.0, 1e-6)])
def test_simulation_summary_matches_oracle(fam, theta, delta):
    g = np.random.default_rng(7 + fam)
    S = 50
    tf = theta + 0.01 * g.standard_normal(S)
    tc = tf + 0.002 * g.standard_normal(S) + 0.001
    out = cg.simulation_summary(fam, torch.from_numpy(tc).cuda(), torch.from_numpy(tf).cuda(), delta)
    out = dict(zip(cg.SIM_SUMMARY, out.cpu().numpy()))
    ref = oracle.simulation_summary(tc, tf)
    for k in ("theta_combined_sim", "theta_full_sim"):
        assert abs(out[k] - ref[k]) <= 1e-14 * abs(ref[k])
    assert abs(out["bias"] - ref["bias"]) <= 1e-12 * abs(ref["bias"]) + 1e-16
    assert abs(out["mse"] - ref["mse"]) <= 1e-12 * ref["mse"]
    d1, d2 = oracle.relative_distances(fam, ref["theta_full_sim"], ref["theta_combined_sim"], delta)
    assert abs(out["d1_relative"] - d1) <= 1e-11 * d1 and abs(out["d2_relative"] - d2) <= 1e-11 * d2


@pytest.mark.parametrize("prec", ["f64", "f32c"])
def test_small_simulation_study_end_to_end(prec):
    """S = 8 replicates of Frank theta = 5 with N = 20,000 pairs and M = 10
    subsets: replicates drawn on the device, the M-subset and full-data fits
    in two batched calls, the summary on the GPU; the oracle fits the same
    replicates (copied to the host) and summarises them.  Agreement is bound
    by the theta bar of the precision (the summary itself is exact up to
    rounding)."""
    fam, theta, N, M, S = 1, 5.0, 20_000, 10, 8
    g = torch.Generator(device="cuda")
    us, vs = [], []
    for s in range(S):
        g.manual_seed(9100 + s)
        u, v = dsyn.sample(fam, theta, N, g)
        us.append(u.float())
        vs.append(v.float())
    u, v = torch.cat(us), torch.cat(vs)
    dofs = np.arange(S + 1, dtype=np.int64) * N
    sub = np.concatenate([[0]] + [cs.equal_offsets(N, M)[1:] + s * N for s in range(S)]).astype(np.int64)
    r_sub = cg.fit_batch(u, v, [fam] * S, dofs, sub, np.arange(S + 1, dtype=np.int64) * M, prec)
    r_full = cg.fit_batch(u, v, [fam] * S, dofs, dofs, np.arange(S + 1, dtype=np.int64), prec)
    out = dict(zip(cg.SIM_SUMMARY, cg.simulation_summary(fam, r_sub.combined, r_full.theta).cpu().numpy()))
    hu, hv = u.cpu().numpy(), v.cpu().numpy()
    oc, of = [], []
    for s in range(S):
        sl = slice(s * N, (s + 1) * N)
        oc.append(oracle.fit(fam, hu[sl], hv[sl], cs.equal_offsets(N, M), nthreads=os.cpu_count() or 1)["combined"])
        of.append(oracle.fit(fam, hu[sl], hv[sl], np.array([0, N]))["theta"][0])
    ref = oracle.simulation_summary(oc, of)
    tol = {"f64": 1e-9, "f32c": 1e-5}[prec]
    assert abs(out["theta_combined_sim"] - ref["theta_combined_sim"]) <= tol * theta
    assert abs(out["theta_full_sim"] - ref["theta_full_sim"]) <= tol * theta
    assert abs(out["bias"] - ref["bias"]) <= 2 * tol * theta
    d1, d2 = oracle.relative_distances(fam, ref["theta_full_sim"], ref["theta_combined_sim"], 0.0)
    assert np.isfinite(out["d1_relative"]) and out["d1_relative"] > 0
    # the distances follow the bias: relative agreement within the theta bar
    # amplified by |bias| / theta
    amp = theta / max(abs(ref["bias"]), 1e-12)
    assert abs(out["d1_relative"] - d1) <= 4 * tol * amp * d1
    assert abs(out["d2_relative"] - d2) <= 4 * tol * amp * d2
