"""Batched path: a CUDA-graph-captured plan over a mixed batch of datasets
(family uniform over the three, tau in [0.1, 0.8], n log-uniform), replayed
on new data; the autotuned block table; and the full-size 4096-dataset batch
checked against the oracle on sampled datasets."""
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


def _err(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)) / np.maximum(np.abs(np.asarray(b)), 0.05)


@pytest.mark.parametrize("prec", ["f32c", "f64"])
def test_graph_replay_equals_direct_fit_and_follows_new_data(prec):
    bt = dsyn.mixed_batch(B=48, seed=77, n_lo=1e3, n_hi=1e5)
    plan = cg.BatchPlan(bt["families"], bt["dataset_offsets"], bt["subset_offsets"], bt["dataset_subset_start"],
                        precision=prec)
    u, v = bt["u"].clone(), bt["v"].clone()
    g = plan.capture(u, v)
    g.replay()
    torch.cuda.synchronize()
    direct = cg.fit_batch(bt["u"], bt["v"], bt["families"], bt["dataset_offsets"], bt["subset_offsets"],
                          bt["dataset_subset_start"], prec)
    assert torch.equal(plan.theta, direct.theta) and torch.equal(plan.combined, direct.combined)
    # new data in the same buffers: the replay follows it
    bt2 = dsyn.mixed_batch(B=48, seed=77, n_lo=1e3, n_hi=1e5)  # same shapes/families
    g2 = torch.Generator(device="cuda")
    g2.manual_seed(5)
    perm = torch.randperm(u.shape[0], generator=g2, device="cuda")
    u.copy_(bt2["u"][perm])
    v.copy_(bt2["v"][perm])
    g.replay()
    torch.cuda.synchronize()
    direct2 = cg.fit_batch(u, v, bt["families"], bt["dataset_offsets"], bt["subset_offsets"],
                           bt["dataset_subset_start"], prec)
    assert torch.equal(plan.theta, direct2.theta)
    plan.close()


def test_block_table_changes_blocks_not_results_beyond_rounding():
    bt = dsyn.mixed_batch(B=24, seed=78, n_lo=5e3, n_hi=2e5)
    args = (bt["u"], bt["v"], bt["families"], bt["dataset_offsets"], bt["subset_offsets"], bt["dataset_subset_start"])
    ctx = cg.Context()
    a = cg.fit_batch(*args, "f32c", ctx=ctx)
    cg.set_blocks([(20480, 256)], ctx)
    b = cg.fit_batch(*args, "f32c", ctx=ctx)
    cg.set_blocks([], ctx)
    c = cg.fit_batch(*args, "f32c", ctx=ctx)
    assert torch.equal(a.theta, c.theta)
    assert _err(b.theta.cpu().numpy(), a.theta.cpu().numpy()).max() <= 1e-5


def _replay_ms(plan, u, v, reps=7):
    g = plan.capture(u, v)
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def test_autotuner_tables_are_valid_per_family_and_no_slower_than_default():
    """Per-family tables of valid blocks (or [] for the built-in rule), each
    the fastest of its candidates on the family's mixed-size batch; installed
    on a context, they fit a mixed batch of all three families no slower than
    the built-in rule (within timing noise), with results within the
    precision's bar of the rule's."""
    from paper_1609_05530_gb300 import autotune
    tables = autotune.tune("f32c", "f32", reps=3)
    assert set(tables) == {cg.GAUSSIAN, cg.FRANK, cg.GUMBEL}
    for fam, (table, timings) in tables.items():
        assert [] in [t["table"] for t in timings]           # the built-in rule was a candidate
        assert min(t["ms"] for t in timings) == next(t["ms"] for t in timings if t["table"] == table)
        assert all(b in (128, 256, 512) for _, b in table)
        assert [m for m, _ in table] == sorted(m for m, _ in table)
        assert not table or table[-1][0] >= 20480
    bt = dsyn.mixed_batch(B=512, seed=81, n_lo=2e3, n_hi=4e5)
    args = (bt["families"], bt["dataset_offsets"], bt["subset_offsets"], bt["dataset_subset_start"])
    ctx0 = cg.Context()
    base = cg.BatchPlan(*args, precision="f32c", ctx=ctx0)
    t_default = _replay_ms(base, bt["u"], bt["v"])
    ctx = cg.Context()
    for fam, (table, _) in tables.items():
        cg.set_blocks(table, ctx, family=fam)
    tuned = cg.BatchPlan(*args, precision="f32c", ctx=ctx)
    t_tuned = _replay_ms(tuned, bt["u"], bt["v"])
    assert t_tuned <= 1.05 * t_default, (t_tuned, t_default)
    assert _err(tuned.theta.cpu().numpy(), base.theta.cpu().numpy()).max() <= 1e-5
    base.close()
    tuned.close()


@pytest.mark.parametrize("prec", ["f32c", "f64"])
def test_full_mixed_batch_4096_datasets_sampled_against_oracle(prec):
    bt = dsyn.mixed_batch(B=4096)
    n = int(bt["dataset_offsets"][-1])
    assert 4e8 < n < 8e8
    plan = cg.BatchPlan(bt["families"], bt["dataset_offsets"], bt["subset_offsets"], bt["dataset_subset_start"],
                        precision=prec)
    g = plan.capture(bt["u"], bt["v"])
    g.replay()
    torch.cuda.synchronize()
    th, comb, st = plan.theta.cpu().numpy(), plan.combined.cpu().numpy(), plan.status.cpu().numpy()
    assert np.isfinite(comb).all()
    rng = np.random.default_rng(0)
    dofs, soff, dss = bt["dataset_offsets"], bt["subset_offsets"], bt["dataset_subset_start"]
    sizes = np.diff(dofs)
    pick = list(rng.choice(4096, 40, replace=False)) + [int(np.argmax(sizes)), int(np.argmin(sizes))]
    for b in pick:
        lo, hi = int(dofs[b]), int(dofs[b + 1])
        u = bt["u"][lo:hi].cpu().numpy()
        v = bt["v"][lo:hi].cpu().numpy()
        off = soff[dss[b]:dss[b + 1] + 1] - lo
        o = oracle.fit(int(bt["families"][b]), u, v, off, nthreads=os.cpu_count() or 1)
        sl = slice(dss[b], dss[b + 1])
        assert np.array_equal(st[sl], o["status"]), b
        assert _err(th[sl], o["theta"]).max() <= THETA_TOL[prec], b
        assert _err(comb[b], o["combined"]) <= THETA_TOL[prec], b
    plan.close()


@pytest.mark.parametrize("pinned", [True, False])
def test_batch_host_buffers_equal_device_batch(pinned):
    """copula_fit_batch_host (host columns in, host results out; pinned inputs
    read in place, pageable ones copied) gives the bits of copula_fit_batch."""
    bt = dsyn.mixed_batch(B=40, seed=79, n_lo=1e3, n_hi=3e5)
    args = (bt["families"], bt["dataset_offsets"], bt["subset_offsets"], bt["dataset_subset_start"])
    ctx = cg.Context()
    d = cg.fit_batch(bt["u"], bt["v"], *args, "f32c", ctx=ctx)
    if pinned:
        hu, hv = bt["u"].cpu().pin_memory(), bt["v"].cpu().pin_memory()
    else:
        hu, hv = bt["u"].cpu().numpy(), bt["v"].cpu().numpy()
    th, var, st, comb = cg.fit_batch_host(hu, hv, *args, "f32c", ctx=ctx)
    assert np.array_equal(th, d.theta.cpu().numpy())
    assert np.array_equal(var, d.var.cpu().numpy())
    assert np.array_equal(st, d.status.cpu().numpy())
    assert np.array_equal(comb, d.combined.cpu().numpy())


def test_plan_diagnostics_report_the_passes_of_each_subset():
    bt = dsyn.mixed_batch(B=12, seed=80, n_lo=2e3, n_hi=1e5)
    dofs, soff, dss = bt["dataset_offsets"], bt["subset_offsets"], bt["dataset_subset_start"]
    ctx = cg.Context()
    plan = cg.BatchPlan(bt["families"], dofs, soff, dss, precision="f32c", ctx=ctx)
    plan.run(bt["u"], bt["v"])
    info, iters = plan.diagnostics()
    torch.cuda.synchronize()
    info, iters = info.cpu().numpy(), iters.cpu().numpy()
    for b in range(12):
        lo, hi = int(dofs[b]), int(dofs[b + 1])
        r, dg = cg.fit_ex(bt["u"][lo:hi], bt["v"][lo:hi], soff[dss[b]:dss[b + 1] + 1] - lo, int(bt["families"][b]),
                          "f32c", ctx=ctx)
        sl = slice(dss[b], dss[b + 1])
        assert np.array_equal(iters[sl], dg.iters.cpu().numpy()), b
        assert np.array_equal(info[sl], dg.info.cpu().numpy()), b
        if bt["families"][b] != 0:
            assert (iters[sl] >= 1).all()
    plan.close()


def test_unit_rates_are_measured_and_plausible():
    r = cg.measure_unit_rates()
    assert set(r) == set(cg.UNIT_RATES)
    # MUFU: a few per SM per clock; FP32 FMA: about 128 per SM per clock;
    # FP64 FMA: far below FP32 on this GPU
    assert 5e11 < r["mufu_ex2"] < 5e13 and 5e11 < r["mufu_lg2"] < 5e13 and 5e11 < r["mufu_rcp"] < 5e13
    assert 5e12 < r["fp32_fma"] < 1e15 and r["fp32_fma"] > 2 * r["mufu_ex2"]
    assert 1e9 < r["fp64_fma"] < r["fp32_fma"]
