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


def test_autotuner_produces_a_valid_table():
    from paper_1609_05530_gb300 import autotune
    ctx = cg.Context()
    table, timings = autotune.tune("f32c", "f32", reps=2, ctx=ctx)
    assert table and all(b in (128, 256, 512) for _, b in table)
    assert [m for m, _ in table] == sorted(m for m, _ in table) and table[-1][0] >= 20480
    cg.set_blocks(table, ctx)


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
    pick = list(rng.choice(4096, 10, replace=False)) + [int(np.argmax(sizes)), int(np.argmin(sizes))]
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
