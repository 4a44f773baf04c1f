"""FP64 CPU oracle of the divide-and-combine MPL copula estimator -- TEST INFRASTRUCTURE.

This package is the plain, slow reference that the CUDA library is checked
against (Wei, Kim & Conlon, arXiv:1609.05530: Eq. 12 ranks, Eq. 13 pseudo
log-likelihood, Eq. 14 row partition, Eq. 15 inverse-variance combine, and the
Genest-Ghoudi-Rivest sandwich variance cited in Section 2.3).  Only the
test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA path, and the
CUDA path never imports it.

The arithmetic lives in ``copula_oracle.c`` (plain C, FP64); this module
compiles it with gcc on first use and wraps it with ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

GAUSSIAN, FRANK, GUMBEL = 0, 1, 2
FAMILIES = {"gaussian": GAUSSIAN, "frank": FRANK, "gumbel": GUMBEL}
DTYPE_F32, DTYPE_F64 = 0, 1
W_INVVAR, W_FISHER, W_EQUAL = 0, 1, 2
OK, BOUNDARY, NOT_CONVERGED, DEGENERATE, CAPPED = 0, 1, 2, 3, 4

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "copula_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

_d = ctypes.c_double
_i64 = ctypes.c_int64
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile ``copula_oracle.c`` into ``_build/liboracle.so`` (gcc, -O2, IEEE FP)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=gnu11", "-o", tmp, _SRC,
                               "-lm", "-lpthread"])
        os.replace(tmp, _OUT)
    return _OUT


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_ndtri_lower.restype = _d
            L.orc_ndtri_lower.argtypes = [_d]
            L.orc_ranks.argtypes = [ctypes.c_int, _vp, _i64, _i64p, _i64, _i32p]
            L.orc_point.argtypes = [ctypes.c_int, _d, _i64, _i64, _i64, _dp]
            L.orc_terms_at.argtypes = [ctypes.c_int, _d, _d, _d, _dp]
            L.orc_terms_at.restype = None
            L.orc_density_vec.argtypes = [ctypes.c_int, _d, _dp, _dp, _i64, _dp]
            L.orc_density_vec.restype = None
            L.orc_cdf.restype = _d
            L.orc_cdf.argtypes = [ctypes.c_int, _d, _d, _d]
            L.orc_loglik.argtypes = [ctypes.c_int, _d, _i32p, _i32p, _i64, _dp, _dp, _dp]
            L.orc_var_at.restype = _d
            L.orc_var_at.argtypes = [ctypes.c_int, _d, _i32p, _i32p, _i64, ctypes.c_int]
            L.orc_fit_ranks.argtypes = [ctypes.c_int, _i32p, _i32p, _i64, _dp, _dp, _dp,
                                        ctypes.POINTER(ctypes.c_int)]
            L.orc_combine.restype = _d
            L.orc_combine.argtypes = [_dp, _dp, _dp, _i32p, _i64, ctypes.c_int]
            L.orc_fit.argtypes = [ctypes.c_int, ctypes.c_int, _vp, _vp, _i64, _i64p, _i64,
                                  ctypes.c_int, _dp, _dp, _dp, _i32p, _i32p, _dp, ctypes.c_int]
            for f in (L.orc_kendall_tau, L.orc_kendall_tau_merge, L.orc_spearman_rho):
                f.restype = _d
                f.argtypes = [_i32p, _i32p, _i64]
            for f in (L.orc_tau_of_theta, L.orc_rho_s_of_theta):
                f.restype = _d
                f.argtypes = [ctypes.c_int, _d]
            L.orc_theta_from_rank_corr.argtypes = [ctypes.c_int, ctypes.c_int, _d, _dp]
            L.orc_density_distance.argtypes = [ctypes.c_int, _d, _d, _d, _dp]
            L.orc_subset_new.restype = _vp
            L.orc_subset_new.argtypes = [ctypes.c_int, _i32p, _i32p, _i64]
            L.orc_subset_sums.restype = None
            L.orc_subset_sums.argtypes = [_vp, _d, _dp, _dp, _dp]
            L.orc_subset_delete.restype = None
            L.orc_subset_delete.argtypes = [_vp]
            _lib = L
    return _lib


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _family(f) -> int:
    return FAMILIES[f] if isinstance(f, str) else int(f)


def ndtri_lower(p: float) -> float:
    """Standard normal quantile for p in (0, 0.5]."""
    return lib().orc_ndtri_lower(float(p))


def ranks(x: np.ndarray, offsets) -> np.ndarray:
    """Within-subset ordinal ranks 1..m (Eq. 12, ties by index); raises on NaN."""
    x = np.ascontiguousarray(x)
    dt = {np.dtype(np.float32): DTYPE_F32, np.dtype(np.float64): DTYPE_F64}[x.dtype]
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    out = np.zeros(x.shape[0], dtype=np.int32)
    rc = lib().orc_ranks(dt, x.ctypes.data, x.shape[0], _ptr(off, _i64p), off.shape[0] - 1,
                         _ptr(out, _i32p))
    if rc != 0:
        raise ValueError("NaN in input")
    return out


def point(family, theta: float, ru: int, rv: int, m: int) -> np.ndarray:
    """[l, l_t, l_tt, l_tu, l_tv] at the pseudo-observation (ru/(m+1), rv/(m+1))."""
    out = np.zeros(5)
    if lib().orc_point(_family(family), float(theta), int(ru), int(rv), int(m), _ptr(out, _dp)):
        raise ValueError("bad point")
    return out


def terms_at(family, theta: float, u: float, v: float) -> np.ndarray:
    """[l, l_t, l_tt, l_tu, l_tv] at an arbitrary (u, v) in (0,1)^2."""
    out = np.zeros(5)
    lib().orc_terms_at(_family(family), float(theta), float(u), float(v), _ptr(out, _dp))
    return out


def density(family, theta: float, u, v) -> np.ndarray:
    """Copula density c(u, v; theta) at arrays of points."""
    u = np.ascontiguousarray(u, dtype=np.float64).ravel()
    v = np.ascontiguousarray(v, dtype=np.float64).ravel()
    out = np.empty_like(u)
    lib().orc_density_vec(_family(family), float(theta), _ptr(u, _dp), _ptr(v, _dp), u.shape[0],
                          _ptr(out, _dp))
    return out


def cdf(family, theta: float, u: float, v: float) -> float:
    return lib().orc_cdf(_family(family), float(theta), float(u), float(v))


def loglik(family, theta: float, ru: np.ndarray, rv: np.ndarray):
    """(l, g, h): Eq. 13 and its theta-derivatives summed over one subset."""
    ru = np.ascontiguousarray(ru, dtype=np.int32)
    rv = np.ascontiguousarray(rv, dtype=np.int32)
    l, g, h = _d(), _d(), _d()
    lib().orc_loglik(_family(family), float(theta), _ptr(ru, _i32p), _ptr(rv, _i32p), ru.shape[0],
                     ctypes.byref(l), ctypes.byref(g), ctypes.byref(h))
    return l.value, g.value, h.value


class Subset:
    """One subset's per-point margin transforms, built once from its ranks
    (orc_subset_new), on which Eq. 13 passes can then be run one at a time
    (orc_subset_sums): the transform and pass stages of a fit, apart."""

    def __init__(self, family, ru, rv):
        self._ru = np.ascontiguousarray(ru, dtype=np.int32)
        self._rv = np.ascontiguousarray(rv, dtype=np.int32)
        self.m = self._ru.shape[0]
        self._h = lib().orc_subset_new(_family(family), _ptr(self._ru, _i32p), _ptr(self._rv, _i32p), self.m)
        if not self._h:
            raise ValueError("bad subset")

    def sums(self, theta: float):
        """(l, g, h) of Eq. 13 at theta over the subset."""
        l, g, h = _d(), _d(), _d()
        lib().orc_subset_sums(self._h, float(theta), ctypes.byref(l), ctypes.byref(g), ctypes.byref(h))
        return l.value, g.value, h.value

    def close(self):
        if self._h:
            lib().orc_subset_delete(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def var_at(family, theta: float, ru, rv, direct: bool) -> float:
    """Var(theta_hat) = sigma^2/m of one subset at theta (direct: O(m^2) form)."""
    ru = np.ascontiguousarray(ru, dtype=np.int32)
    rv = np.ascontiguousarray(rv, dtype=np.int32)
    return lib().orc_var_at(_family(family), float(theta), _ptr(ru, _i32p), _ptr(rv, _i32p),
                            ru.shape[0], int(bool(direct)))


def fit_ranks(family, ru, rv):
    """(theta_hat, var, info, status, iters) for one subset given its ranks."""
    ru = np.ascontiguousarray(ru, dtype=np.int32)
    rv = np.ascontiguousarray(rv, dtype=np.int32)
    th, var, info, it = _d(), _d(), _d(), ctypes.c_int()
    st = lib().orc_fit_ranks(_family(family), _ptr(ru, _i32p), _ptr(rv, _i32p), ru.shape[0],
                             ctypes.byref(th), ctypes.byref(var), ctypes.byref(info),
                             ctypes.byref(it))
    return th.value, var.value, info.value, st, it.value


def combine(theta, var, info, status, weight=W_INVVAR) -> float:
    """Eq. 15 in subset order."""
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    var = np.ascontiguousarray(var, dtype=np.float64)
    info = np.ascontiguousarray(info, dtype=np.float64)
    status = np.ascontiguousarray(status, dtype=np.int32)
    return lib().orc_combine(_ptr(theta, _dp), _ptr(var, _dp), _ptr(info, _dp), _ptr(status, _i32p),
                             theta.shape[0], int(weight))


def fit(family, u: np.ndarray, v: np.ndarray, offsets, weight=W_INVVAR, nthreads: int = 1) -> dict:
    """Whole estimator: per-subset MPL fits (Eq. 12-13) and the Eq. 15 combine.

    ``u``/``v`` are float32 or float64 arrays of the raw pair values; ``offsets``
    holds K+1 int64 row offsets (Eq. 14).  Returns theta, var, info (observed
    information -sum l_tt), status, iters per subset and the combined estimate.
    """
    u = np.ascontiguousarray(u)
    v = np.ascontiguousarray(v)
    assert u.dtype == v.dtype and u.shape == v.shape
    dt = {np.dtype(np.float32): DTYPE_F32, np.dtype(np.float64): DTYPE_F64}[u.dtype]
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    K = off.shape[0] - 1
    theta = np.zeros(K)
    var = np.zeros(K)
    info = np.zeros(K)
    status = np.zeros(K, dtype=np.int32)
    iters = np.zeros(K, dtype=np.int32)
    comb = _d()
    rc = lib().orc_fit(_family(family), dt, u.ctypes.data, v.ctypes.data, u.shape[0],
                       _ptr(off, _i64p), K, int(weight), _ptr(theta, _dp), _ptr(var, _dp),
                       _ptr(info, _dp), _ptr(status, _i32p), _ptr(iters, _i32p), ctypes.byref(comb),
                       int(nthreads))
    if rc != 0:
        raise ValueError("invalid arguments to oracle fit")
    return dict(theta=theta, var=var, info=info, status=status, iters=iters, combined=comb.value)


# ---------------------------------------------------------------------------
# Rank-correlation inversion estimators (Section 2.3 lists them beside the MPL)
# ---------------------------------------------------------------------------

def kendall_tau(ru, rv) -> float:
    """Kendall's tau of one subset from its ranks (every pair compared)."""
    ru = np.ascontiguousarray(ru, dtype=np.int32)
    rv = np.ascontiguousarray(rv, dtype=np.int32)
    return lib().orc_kendall_tau(_ptr(ru, _i32p), _ptr(rv, _i32p), ru.shape[0])


def kendall_tau_merge(ru, rv) -> float:
    """Kendall's tau of one subset by counting the inversions of its v-ranks
    in u-rank order with a merge sort (O(m log m); for large subsets)."""
    ru = np.ascontiguousarray(ru, dtype=np.int32)
    rv = np.ascontiguousarray(rv, dtype=np.int32)
    return lib().orc_kendall_tau_merge(_ptr(ru, _i32p), _ptr(rv, _i32p), ru.shape[0])


def spearman_rho(ru, rv) -> float:
    """Spearman's rho of one subset from its ranks, 1 - 6 sum d^2 / (m (m^2 - 1))."""
    ru = np.ascontiguousarray(ru, dtype=np.int32)
    rv = np.ascontiguousarray(rv, dtype=np.int32)
    return lib().orc_spearman_rho(_ptr(ru, _i32p), _ptr(rv, _i32p), ru.shape[0])


def tau_of_theta(family, theta: float) -> float:
    """Population Kendall's tau of the family at theta."""
    return lib().orc_tau_of_theta(_family(family), float(theta))


def rho_s_of_theta(family, theta: float) -> float:
    """Population Spearman's rho of the family at theta."""
    return lib().orc_rho_s_of_theta(_family(family), float(theta))


def theta_from_tau(family, tau: float):
    """(theta, status): the parameter whose population Kendall's tau is tau."""
    th = _d()
    st = lib().orc_theta_from_rank_corr(_family(family), 0, float(tau), ctypes.byref(th))
    return th.value, st


def theta_from_rho_s(family, rho: float):
    """(theta, status): the parameter whose population Spearman's rho is rho."""
    th = _d()
    st = lib().orc_theta_from_rank_corr(_family(family), 1, float(rho), ctypes.byref(th))
    return th.value, st


# ---------------------------------------------------------------------------
# Section 2.5-2.6: the simulation study's summaries (Eq. 16-20)
# ---------------------------------------------------------------------------

def density_integrals(family, theta_a: float, theta_b: float, delta: float = 0.0) -> np.ndarray:
    """Integrals over [delta, 1-delta]^2 of |ca-cb|, |ca|, (ca-cb)^2, ca^2."""
    out = np.zeros(4)
    rc = lib().orc_density_distance(_family(family), float(theta_a), float(theta_b), float(delta),
                                    _ptr(out, _dp))
    if rc == -2:
        raise ValueError("an integrand is not finite at this delta (Gumbel: delta^theta underflows)")
    if rc:
        raise ValueError("bad arguments")
    return out


def relative_distances(family, theta_full: float, theta_combined: float, delta: float = 0.0):
    """(d1, d2): Eq. 19 and Eq. 20 between the densities at the full-data and
    the combined parameter, integrated over [delta, 1-delta]^2."""
    s = density_integrals(family, theta_full, theta_combined, delta)
    return s[0] / s[1], float(np.sqrt(s[2] / s[3]))


def simulation_summary(theta_combined, theta_full) -> dict:
    """Eq. 17 and 18 (means over the S simulations) and the estimated bias and
    MSE of Section 2.6 from per-simulation combined and full-data estimates."""
    tc = np.asarray(theta_combined, dtype=np.float64)
    tf = np.asarray(theta_full, dtype=np.float64)
    comb_sim = float(tc.sum() / tc.shape[0])   # Eq. 17
    full_sim = float(tf.sum() / tf.shape[0])   # Eq. 18
    return dict(theta_combined_sim=comb_sim, theta_full_sim=full_sim, bias=comb_sim - full_sim,
                mse=float(((tc - tf) ** 2).sum() / tc.shape[0]))
