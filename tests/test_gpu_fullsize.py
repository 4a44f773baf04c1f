"""Every subset of the two largest workloads against the oracle, by checks
the oracle makes one subset at a time at any size (Section 2.3, Eq. 12-13):

- the ranks of both columns (Eq. 12) equal the oracle's, bit for bit (the
  streaming sample sort for the large Gumbel subsets, the shared-memory
  ordering for the others);
- each estimate with status OK is a root of the oracle's own score of
  Eq. 13 on those ranks: the Newton step -g/h the oracle takes from the
  GPU's estimate stays within the precision's theta bar;
- each variance equals the oracle's sandwich variance at the GPU's
  estimate, within the precision's variance bar;
- each other status (BOUNDARY, CAPPED, NOT_CONVERGED) is the oracle's
  status for that subset, with its estimate within the bar.

Gumbel theta = 2, n = 1e8, K = 1000 lognormal sizes (875 subsets on the
streaming path), and the 4096-dataset batch (60,729 subsets).  The oracle's
calls run on the host cores in threads (its C routines release the
interpreter lock)."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1609_05530_gb300 as cg  # noqa: E402
from copula_synth import device as dsyn  # noqa: E402

NCPU = os.cpu_count() or 1
THETA_TOL = {"f64": 1e-9, "f32c": 1e-5}
VAR_TOL = {"f64": 1e-8, "f32c": 2e-4}


def oracle_ranks(x, off):
    """The oracle's ranks of every subset, the subsets split into runs of
    about equal size over the host threads."""
    K = len(off) - 1
    out = np.empty(x.shape[0], dtype=np.int32)
    cuts = np.searchsorted(off, np.linspace(0, off[-1], 4 * NCPU + 1), side="left")
    cuts = np.unique(np.clip(cuts, 0, K))
    if cuts[0] != 0:
        cuts = np.concatenate([[0], cuts])
    if cuts[-1] != K:
        cuts = np.concatenate([cuts, [K]])

    def run(a, b):
        lo, hi = int(off[a]), int(off[b])
        out[lo:hi] = oracle.ranks(x[lo:hi], off[a:b + 1] - lo)

    with ThreadPoolExecutor(NCPU) as ex:
        list(ex.map(lambda ab: run(*ab), zip(cuts[:-1], cuts[1:])))
    return out


def check_every_subset(fam_of, off, hu, hv, ru_gpu, rv_gpu, theta, var, status, prec):
    """Ranks equal; OK estimates are roots of the oracle's score with the
    oracle's variance there; other statuses agree with the oracle's fit."""
    ru, rv = oracle_ranks(hu, off), oracle_ranks(hv, off)
    assert np.array_equal(ru_gpu, ru)
    assert np.array_equal(rv_gpu, rv)
    K = len(off) - 1
    tol = THETA_TOL[prec]

    def step(k):
        lo, hi = int(off[k]), int(off[k + 1])
        th = float(theta[k])
        if status[k] != cg.OK:
            o = oracle.fit(int(fam_of[k]), hu[lo:hi], hv[lo:hi], np.array([0, hi - lo]))
            return k, int(o["status"][0]), abs(th - o["theta"][0]) / max(abs(o["theta"][0]), 0.05), 0.0
        f = int(fam_of[k])
        _, g, h = oracle.loglik(f, th, ru[lo:hi], rv[lo:hi])
        ov = oracle.var_at(f, th, ru[lo:hi], rv[lo:hi], False)
        return (k, cg.OK, abs(g / h) / max(abs(th), 0.05) if h < 0 else np.inf,
                abs(float(var[k]) - ov) / ov)

    with ThreadPoolExecutor(NCPU) as ex:
        res = list(ex.map(step, range(K)))
    worst = max(res, key=lambda r: r[2])
    worst_var = max(res, key=lambda r: r[3])
    assert all(r[1] == status[r[0]] for r in res), [r for r in res if r[1] != status[r[0]]][:5]
    print(f"{prec}: {K} subsets, worst theta step {worst[2]:.3e} (subset {worst[0]}), worst variance "
          f"{worst_var[3]:.3e} (subset {worst_var[0]}), {int((status != cg.OK).sum())} not OK")
    assert worst[2] <= tol, worst
    assert worst_var[3] <= VAR_TOL[prec], worst_var


@pytest.fixture(scope="module")
def gumbel_1e8():
    u, v, off = dsyn.gumbel_lognormal()
    hu, hv = u.cpu().numpy(), v.cpu().numpy()
    ru = cg.ranks(u, off).cpu().numpy()
    rv = cg.ranks(v, off).cpu().numpy()
    yield u, v, off, hu, hv, ru, rv
    del u, v
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", ["f32c", "f64"])
def test_gumbel_1e8_every_subset_against_the_oracle(prec, gumbel_1e8):
    u, v, off, hu, hv, ru, rv = gumbel_1e8
    r = cg.fit(u, v, off, cg.GUMBEL, prec)
    th, var, st = r.theta.cpu().numpy(), r.var.cpu().numpy(), r.status.cpu().numpy()
    assert (np.diff(off) > cg.MAX_SUBSET).sum() > 800  # most subsets on the streaming path
    fam = np.full(len(off) - 1, cg.GUMBEL)
    check_every_subset(fam, off, hu, hv, ru, rv, th, var, st, prec)


@pytest.fixture(scope="module")
def mixed_4096():
    bt = dsyn.mixed_batch(B=4096)
    soff = bt["subset_offsets"]
    hu, hv = bt["u"].cpu().numpy(), bt["v"].cpu().numpy()
    ru = cg.ranks(bt["u"], soff).cpu().numpy()
    rv = cg.ranks(bt["v"], soff).cpu().numpy()
    fam_of = np.repeat(bt["families"], np.diff(bt["dataset_subset_start"]))
    yield bt, hu, hv, ru, rv, fam_of
    del bt
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", ["f32c", "f64"])
def test_mixed_4096_every_subset_against_the_oracle(prec, mixed_4096):
    bt, hu, hv, ru, rv, fam_of = mixed_4096
    r = cg.fit_batch(bt["u"], bt["v"], bt["families"], bt["dataset_offsets"], bt["subset_offsets"],
                     bt["dataset_subset_start"], prec)
    th, var, st = r.theta.cpu().numpy(), r.var.cpu().numpy(), r.status.cpu().numpy()
    assert len(th) == 60_729
    check_every_subset(fam_of, bt["subset_offsets"], hu, hv, ru, rv, th, var, st, prec)
