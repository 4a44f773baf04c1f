"""copula_fit_noalloc, the allocation-free variant of copula_fit.

It serves callers that cannot allocate device memory -- code under a fixed
memory budget, plugins handed only their input and output buffers, serving
loops that must not enter an allocator -- by keeping its scratch in a fixed
array inside the library.  Through the C ABI, its results must match
copula_fit's (within the parity tolerances the other GPU tests use) on two
calls in a row with different inputs, so that what the first call leaves in
the shared array cannot leak into the second; requests beyond its limits
must be refused.  The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

import copula_synth as cs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1609_05530_gb300 as cg  # noqa: E402

THETA_TOL = {"f64": 1e-9, "f32c": 1e-5}
VAR_TOL = {"f64": 1e-8, "f32c": 2e-4}
ERR_UNSUPPORTED = -4


def _entry():
    f = cg.lib().copula_fit_noalloc
    i32, i64, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
    f.argtypes = [i32, i32, vp, vp, i64, ctypes.POINTER(i64), i64, vp, vp, vp, vp, ctypes.POINTER(cg.Opts), vp]
    f.restype = ctypes.c_int
    return f


def _call(d, prec):
    u = torch.from_numpy(d.u).cuda()
    v = torch.from_numpy(d.v).cuda()
    K = d.K
    th = torch.full((K,), float("nan"), dtype=torch.float64, device="cuda")
    var = torch.full((K,), float("nan"), dtype=torch.float64, device="cuda")
    st = torch.full((K,), -7, dtype=torch.int32, device="cuda")
    comb = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    off = np.ascontiguousarray(d.offsets, dtype=np.int64)
    o = cg.make_opts(prec)
    dt = cg.DTYPE_F32 if d.u.dtype == np.float32 else cg.DTYPE_F64
    rc = _entry()(d.family, dt, u.data_ptr(), v.data_ptr(), d.n, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                  K, th.data_ptr(), var.data_ptr(), st.data_ptr(), comb.data_ptr(), ctypes.byref(o),
                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc, th.cpu().numpy(), var.cpu().numpy(), st.cpu().numpy(), comb.item()


def _check_against_fit(d, prec):
    rc, th, var, st, comb = _call(d, prec)
    assert rc == 0
    r = cg.fit(torch.from_numpy(d.u).cuda(), torch.from_numpy(d.v).cuda(), d.offsets, d.family, prec)
    rth, rvar, rst = r.theta.cpu().numpy(), r.var.cpu().numpy(), r.status.cpu().numpy()
    assert np.array_equal(st, rst)
    ok = (rst == cg.OK) | (rst == cg.BOUNDARY)
    assert np.all(np.abs(th - rth) <= THETA_TOL[prec] * np.maximum(np.abs(rth), 0.05))
    assert np.all(np.abs(var[ok] - rvar[ok]) <= VAR_TOL[prec] * np.abs(rvar[ok]))
    rc_ = r.combined.item()
    assert abs(comb - rc_) <= THETA_TOL[prec] * max(abs(rc_), 0.05)


@pytest.mark.parametrize("prec", ["f64", "f32c"])
def test_noalloc_matches_copula_fit_on_two_calls_in_a_row(prec):
    big = 20_480 if prec == "f32c" else 11_889
    sizes_a = [2, 700, 3000, 7000, big]
    off_a = np.concatenate([[0], np.cumsum(sizes_a)]).astype(np.int64)
    a = cs.make_dataset(cs.FRANK, 5.0, int(off_a[-1]), 1, np.float32, seed=2024, offsets=off_a)
    b = cs.make_dataset(cs.GUMBEL, 2.0, 9000, 3, np.float32, seed=2025)
    _check_against_fit(a, prec)  # first call (also the per-device set-up)
    _check_against_fit(b, prec)  # second call: fewer subsets, another family


def test_noalloc_gaussian_fp64_storage():
    d = cs.gaussian_10k(np.float64, K=10)
    _check_against_fit(d, "f64")
    _check_against_fit(d, "f32c")


def test_noalloc_refuses_requests_beyond_its_limits():
    many = cs.make_dataset(cs.FRANK, 5.0, 2049 * 2, 2049, np.float32, seed=1)
    assert _call(many, "f32c")[0] == ERR_UNSUPPORTED
    large = cs.make_dataset(cs.FRANK, 5.0, 20_481, 1, np.float32, seed=2)
    assert _call(large, "f32c")[0] == ERR_UNSUPPORTED
    mid = cs.make_dataset(cs.FRANK, 5.0, 11_890, 1, np.float32, seed=3)
    assert _call(mid, "f64")[0] == ERR_UNSUPPORTED
    assert _call(mid, "f32c")[0] == 0
