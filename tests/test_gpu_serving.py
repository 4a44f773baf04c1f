"""The serving loop: requests of different sizes, families and subset counts,
submitted while others run, are batched together on the GPU; every result
must equal (bitwise) the same dataset fitted alone with copula_fit, and
every served result must match the FP64 CPU oracle's fit of the same data
(theta within 1e-9 relative on the FP64 path and 1e-5 on the FP32C path,
relative to max(|theta|, 0.05); equal statuses; the variance where defined;
Eq. 15 to the theta bar)."""
import os
import threading

import numpy as np
import pytest

import copula_synth as cs
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1609_05530_gb300 as cg  # noqa: E402


def _requests(count, seed):
    g = np.random.default_rng(seed)
    out = []
    for i in range(count):
        fam = int(g.integers(0, 3))
        tau = float(g.uniform(0.1, 0.8))
        n = int(np.exp(g.uniform(np.log(4_000), np.log(300_000))))
        K = max(1, n // 10_000)
        out.append(cs.make_dataset(fam, cs.theta_of_tau(fam, tau), n, K, np.float32, seed=seed * 100 + i))
    return out


THETA_TOL = {"f64": 1e-9, "f32c": 1e-5}
VAR_TOL = {"f64": 1e-8, "f32c": 2e-4}
VAR_MIN_M = {"f64": 16, "f32c": 64}


def _rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), 0.05)


def _check_against_oracle(d, o, prec):
    """One served request against the oracle's fit of its dataset."""
    ref = oracle.fit(d.family, d.u, d.v, d.offsets, nthreads=os.cpu_count() or 1)
    assert np.array_equal(o["status"], ref["status"]), (o["status"], ref["status"])
    ok = ref["status"] != oracle.DEGENERATE
    e = _rel(o["theta"][ok], ref["theta"][ok])
    assert e.max() <= THETA_TOL[prec], (prec, d.family, e.max())
    m = np.diff(d.offsets)
    vok = np.isin(ref["status"], (oracle.OK, oracle.BOUNDARY)) & (m >= VAR_MIN_M[prec])
    if vok.any():
        ve = np.abs(o["var"][vok] - ref["var"][vok]) / np.abs(ref["var"][vok])
        assert ve.max() <= VAR_TOL[prec], (prec, d.family, ve.max())
    assert _rel(o["combined"], ref["combined"]) <= THETA_TOL[prec]


def _solo(d, prec):
    r = cg.fit(torch.from_numpy(d.u).cuda(), torch.from_numpy(d.v).cuda(), d.offsets, d.family, prec)
    return r.theta.cpu().numpy(), r.var.cpu().numpy(), r.status.cpu().numpy(), r.combined.item()


@pytest.mark.parametrize("prec", ["f32c", "f64"])
def test_results_in_the_mix_equal_results_alone(prec):
    # three large requests first, one per stream, so that the small ones
    # arrive while the GPU is busy and must be admitted together
    big = [cs.make_dataset(f, th, 20_000_000, 2000, np.float32, seed=390 + f)
           for f, th in ((0, 0.4), (1, 4.0), (2, 2.0))]
    ds = _requests(14, seed=3)
    srv = cg.Server(4 << 30, max_slots=8, streams=3)
    tb = [srv.submit(d.u, d.v, d.offsets, d.family, prec) for d in big]
    tickets = [srv.submit(d.u, d.v, d.offsets, d.family, prec) for d in ds]
    outs = [srv.wait(t, timeout_s=120) for t in tickets]
    ob = [srv.wait(t, timeout_s=120) for t in tb]
    st = srv.stats()
    srv.close()
    for d, o in zip(big, ob):
        assert o["state"] == cg.REQ_DONE, o
        assert np.array_equal(o["theta"], _solo(d, prec)[0])
    for d, o in zip(ds, outs):
        assert o["state"] == cg.REQ_DONE, o
        th, var, status, comb = _solo(d, prec)
        assert np.array_equal(o["theta"], th)
        assert np.array_equal(o["var"], var)
        assert np.array_equal(o["status"], status)
        assert o["combined"] == comb
        assert 0 <= o["queue_s"] <= o["latency_s"]
        _check_against_oracle(d, o, prec)
    assert st["fits_done"] == len(ds) + len(big) and st["errors"] == 0
    assert st["batches"] >= 2 and st["mean_batch"] > 1.0   # requests really were batched together
    assert 0 < st["p50_s"] <= st["p99_s"]


def test_concurrent_submitters_and_a_tight_budget():
    ds = _requests(10, seed=4)
    need = max(8 * d.n + 64 * d.K for d in ds) * 6          # room for only a few requests at a time
    srv = cg.Server(max(need, 1 << 22), max_slots=4, streams=2)
    tickets = [None] * len(ds)

    def submit(i):
        tickets[i] = srv.submit(ds[i].u, ds[i].v, ds[i].offsets, ds[i].family)

    th = [threading.Thread(target=submit, args=(i,)) for i in range(len(ds))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    outs = [srv.wait(t, timeout_s=120) for t in tickets]
    srv.close()
    for d, o in zip(ds, outs):
        assert o["state"] == cg.REQ_DONE
        assert np.array_equal(o["theta"], _solo(d, "f32c")[0])
        _check_against_oracle(d, o, "f32c")


def test_rejects_requests_larger_than_the_budget():
    d = cs.make_dataset(1, 5.0, 400_000, 40, np.float32, seed=1)   # 3.2 MB of inputs
    srv = cg.Server(1 << 21, max_slots=2, streams=1)                # 2 MiB budget
    with pytest.raises(cg.CopulaError):
        srv.submit(d.u, d.v, d.offsets, d.family)
    srv.close()


@pytest.mark.parametrize("prec", ["f32c", "f64"])
def test_requests_with_streaming_subsets_in_the_mix(prec):
    """Requests whose subsets exceed one thread block (the streaming path),
    batched with small ones, give the same bits as the same fits alone."""
    ds = _requests(6, seed=5)
    ds.insert(2, cs.make_dataset(1, 4.0, 150_000, 2, np.float32, seed=551))   # 2 subsets of 75,000
    ds.append(cs.make_dataset(2, 2.5, 60_000, 1, np.float32, seed=552))       # 1 subset of 60,000
    srv = cg.Server(1 << 30, max_slots=8, streams=3)
    tickets = [srv.submit(d.u, d.v, d.offsets, d.family, prec) for d in ds]
    outs = [srv.wait(t, timeout_s=120) for t in tickets]
    st = srv.stats()
    srv.close()
    for d, o in zip(ds, outs):
        assert o["state"] == cg.REQ_DONE, o
        th, var, status, comb = _solo(d, prec)
        assert np.array_equal(o["theta"], th)
        assert np.array_equal(o["var"], var)
        assert np.array_equal(o["status"], status)
        assert o["combined"] == comb
        _check_against_oracle(d, o, prec)
    assert st["fits_done"] == len(ds) and st["errors"] == 0
