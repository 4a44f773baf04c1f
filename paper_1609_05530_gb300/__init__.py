"""GB300-native divide-and-combine copula estimation (Wei, Kim & Conlon,
arXiv:1609.05530) -- Python binding of libcopula.

Argument marshalling only: every step of the estimator runs in the CUDA
kernels of ``csrc/`` behind the C ABI declared in ``include/copula.h``.
PyTorch supplies device memory and the current stream.  There is no CPU
fallback: if the library cannot be built or loaded, or no CUDA device is
present, the calls raise.
"""
from __future__ import annotations

import ctypes
import threading
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

GAUSSIAN, FRANK, GUMBEL = 0, 1, 2
FAMILIES = {"gaussian": GAUSSIAN, "frank": FRANK, "gumbel": GUMBEL}
DTYPE_F32, DTYPE_F64 = 0, 1
PREC_F64, PREC_F32C = 0, 1
PRECISIONS = {"f64": PREC_F64, "f32c": PREC_F32C}
W_INVVAR, W_FISHER, W_EQUAL = 0, 1, 2
WEIGHTS = {"invvar": W_INVVAR, "fisher": W_FISHER, "equal": W_EQUAL}
OK, BOUNDARY, NOT_CONVERGED, DEGENERATE, CAPPED = 0, 1, 2, 3, 4
MAX_SUBSET = 20480          # largest subset one thread block fits (FP32 storage)
MAX_SUBSET_F64 = 15000      # FP64 storage
MAX_SUBSET_STREAM = 3145728  # largest subset of the streaming path (FP32 storage)
MAX_SUBSET_STREAM_F64 = 2097152

_i32, _i64, _d, _vp, _sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)


class CopulaError(RuntimeError):
    pass


class Opts(ctypes.Structure):
    _fields_ = [("precision", _i32), ("weight", _i32), ("max_iter", _i32), ("block", _i32), ("rtol", _d)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    from .build import LIB
    return LIB


def lib() -> ctypes.CDLL:
    """Loads libcopula.so (building it with nvcc first if it is missing)."""
    global _lib
    L = _lib
    if L is not None:
        return L
    with _lock:
        if _lib is None:
            from .build import build
            L = ctypes.CDLL(build())
            L.copula_opts_default.argtypes = [ctypes.POINTER(Opts)]
            L.copula_opts_default.restype = None
            L.copula_ctx_create.argtypes = [ctypes.POINTER(_vp)]
            L.copula_ctx_destroy.argtypes = [_vp]
            L.copula_last_error.argtypes = [_vp]
            L.copula_last_error.restype = ctypes.c_char_p
            L.copula_version.restype = ctypes.c_int
            L.copula_fit_workspace_size.argtypes = [_vp, _i32, ctypes.POINTER(Opts), _i64p, _i64,
                                                    ctypes.POINTER(_sz)]
            L.copula_fit.argtypes = [_vp, _i32, _i32, _vp, _vp, _i64, _i64p, _i64, _vp, _vp, _vp, _vp,
                                     ctypes.POINTER(Opts), _vp, _sz, _vp]
            L.copula_fit_ex.argtypes = [_vp, _i32, _i32, _vp, _vp, _i64, _i64p, _i64, _vp, _vp, _vp, _vp, _vp,
                                        _vp, _vp, ctypes.POINTER(Opts), _vp, _sz, _vp]
            L.copula_ctx_set_timing.argtypes = [_vp, _i32]
            L.copula_ctx_kernel_ms.argtypes = [_vp, ctypes.POINTER(_d)]
            L.copula_ctx_launches.argtypes = [_vp, ctypes.POINTER(_i32)]
            L.copula_ctx_stage_ms.argtypes = [_vp, ctypes.POINTER(_d)]
            L.copula_ctx_stream_stamps.argtypes = [_vp, ctypes.POINTER(ctypes.c_uint64), _i32, ctypes.POINTER(_i32)]
            L.copula_fit_batch_workspace_size.argtypes = [_vp, _i32, ctypes.POINTER(Opts), _i32, _i32p, _i64p,
                                                          _i64p, _i64p, ctypes.POINTER(_sz)]
            L.copula_fit_batch.argtypes = [_vp, _i32, _i32p, _i32, _vp, _vp, _i64p, _i64p, _i64p, _vp, _vp, _vp,
                                           _vp, ctypes.POINTER(Opts), _vp, _sz, _vp]
            L.copula_fit_host_workspace_size.argtypes = [_vp, _i32, ctypes.POINTER(Opts), _i64p, _i64,
                                                         ctypes.POINTER(_sz)]
            L.copula_fit_host.argtypes = [_vp, _i32, _i32, _vp, _vp, _i64, _i64p, _i64, _vp, _vp, _vp, _vp,
                                          ctypes.POINTER(Opts), _vp, _sz, _vp]
            L.copula_fit_batch_host_workspace_size.argtypes = [_vp, _i32, ctypes.POINTER(Opts), _i32, _i32p,
                                                               _i64p, _i64p, _i64p, ctypes.POINTER(_sz)]
            L.copula_fit_batch_host.argtypes = [_vp, _i32, _i32p, _i32, _vp, _vp, _i64p, _i64p, _i64p, _vp, _vp,
                                                _vp, _vp, ctypes.POINTER(Opts), _vp, _sz, _vp]
            L.copula_measure_unit_rates.argtypes = [ctypes.POINTER(_d), _i32, _vp]
            L.copula_theta_from_rank_corr.argtypes = [_i32, _i32, _vp, _i64, _vp, _vp, _vp]
            L.copula_density_distance_workspace_size.argtypes = [_i32, _d, _i64, ctypes.POINTER(_sz)]
            L.copula_density_distance.argtypes = [_i32, _d, _i64, _vp, _vp, _vp, _vp, _vp, _sz, _vp]
            L.copula_simulation_summary_workspace_size.argtypes = [_i32, _d, ctypes.POINTER(_sz)]
            L.copula_simulation_summary.argtypes = [_i32, _d, _i32, _vp, _vp, _vp, _vp, _sz, _vp]
            L.copula_ranks.argtypes = [_vp, _i32, _vp, _i64, _i64p, _i64, _vp, _vp, _sz, _vp]
            L.copula_rank_corr.argtypes = [_vp, _i32, _vp, _vp, _i64, _i64p, _i64, _vp, _vp, _vp, _sz, _vp]
            L.copula_loglik.argtypes = [_vp, _i32, _i32, _vp, _vp, _i64, _i64p, _i64, _vp, _vp, _vp, _vp,
                                        ctypes.POINTER(Opts), _vp, _sz, _vp]
            _lib = L
    return _lib


_torch_ok = False


def _torch():
    global _torch_ok
    import torch
    if not _torch_ok:
        if not torch.cuda.is_available():
            raise CopulaError("libcopula needs a CUDA device; none is available")
        _torch_ok = True
    return torch


def _family(f) -> int:
    return FAMILIES[f] if isinstance(f, str) else int(f)


def make_opts(precision="f32c", weight="invvar", max_iter: int = 0, block: int = 0, rtol: float = 0.0) -> Opts:
    o = Opts()
    lib().copula_opts_default(ctypes.byref(o))
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.weight = WEIGHTS[weight] if isinstance(weight, str) else int(weight)
    if max_iter:
        o.max_iter = int(max_iter)
    if block:
        o.block = int(block)
    o.rtol = float(rtol) if rtol else (1e-13 if o.precision == PREC_F64 else 1e-6)
    return o


class Context:
    """One libcopula context (host staging + tables) on the current device."""

    def __init__(self):
        _torch()
        self._h = _vp()
        rc = lib().copula_ctx_create(ctypes.byref(self._h))
        if rc != 0:
            raise CopulaError(f"copula_ctx_create failed ({rc})")
        self._ws = None
        self._sizes = {}

    def close(self):
        if self._h:
            lib().copula_ctx_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def check(self, rc: int, what: str):
        if rc != 0:
            msg = lib().copula_last_error(self._h).decode()
            raise CopulaError(f"{what} failed ({rc}): {msg}")

    def set_timing(self, on: bool):
        """Record CUDA events around the fit kernel(s) of every call."""
        self.check(lib().copula_ctx_set_timing(self._h, 1 if on else 0), "copula_ctx_set_timing")

    def set_wait_limit(self, spins: int = 0, phantom_arrivals: int = 0):
        """copula_ctx_set_wait_limit: streaming grid-barrier poll limit and,
        for tests of the give-up path, a phantom arrival."""
        L = lib()
        L.copula_ctx_set_wait_limit.argtypes = [_vp, _i64, _i32]
        self.check(L.copula_ctx_set_wait_limit(self.handle, int(spins), int(phantom_arrivals)),
                   "copula_ctx_set_wait_limit")

    def kernel_ms(self) -> float:
        """Span of the last call's fit kernel(s) on its stream (waits for it)."""
        ms = _d()
        self.check(lib().copula_ctx_kernel_ms(self._h, ctypes.byref(ms)), "copula_ctx_kernel_ms")
        return ms.value

    def stage_ms(self):
        """Streaming-path stage spans of the last timed call (ms): ranks of u,
        ranks of v, pi, fit kernel."""
        ms = (_d * 4)()
        self.check(lib().copula_ctx_stage_ms(self._h, ms), "copula_ctx_stage_ms")
        return list(ms)

    def stream_stamps(self) -> np.ndarray:
        """Streaming fit kernel of the last timed call: nanoseconds from its
        start to the release of each of its grid barriers (one per chunk
        sweep or Newton step)."""
        buf = (ctypes.c_uint64 * 256)()
        n = _i32()
        self.check(lib().copula_ctx_stream_stamps(self._h, buf, 256, ctypes.byref(n)), "copula_ctx_stream_stamps")
        t = np.array(buf[:min(n.value, 256)], dtype=np.int64)
        return t[1:] - t[0] if len(t) else t

    def launches(self) -> int:
        """Kernels launched by the last call."""
        n = _i32()
        self.check(lib().copula_ctx_launches(self._h, ctypes.byref(n)), "copula_ctx_launches")
        return n.value

    def workspace_size(self, query: str, dtype: int, opts: "Opts", off: np.ndarray) -> int:
        """Bytes from the library's workspace-size entry point `query`,
        remembered per (dtype, options, partition): answering it plans the
        whole call again (~10 us for 100 subsets)."""
        key = (query, dtype, bytes(opts), off.tobytes())
        nb = self._sizes.get(key)
        if nb is None:
            n = _sz()
            self.check(getattr(lib(), query)(self._h, dtype, ctypes.byref(opts), off.ctypes.data_as(_i64p),
                                             off.shape[0] - 1, ctypes.byref(n)), query)
            nb = n.value
            if len(self._sizes) >= 16:
                self._sizes.clear()
            self._sizes[key] = nb
        return nb

    def workspace(self, nbytes: int, device):
        torch = _torch()
        if self._ws is None or self._ws.numel() < nbytes or self._ws.device != device:
            self._ws = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)
        assert self._ws.data_ptr() % 256 == 0
        return self._ws


_ctx_local = threading.local()


def context() -> Context:
    c = getattr(_ctx_local, "ctx", None)
    if c is None:
        c = Context()
        _ctx_local.ctx = c
    return c


def _dtype_code(t) -> int:
    torch = _torch()
    if t.dtype == torch.float32:
        return DTYPE_F32
    if t.dtype == torch.float64:
        return DTYPE_F64
    raise CopulaError("u and v must be float32 or float64")


def _offsets(off) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(off, dtype=np.int64))


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


@dataclass
class FitResult:
    theta: object      # [K] float64: theta_hat per subset (Eq. 13)
    var: object        # [K] float64: asymptotic variance per subset
    status: object     # [K] int32
    combined: object   # [1] float64: Eq. 15


def fit(u, v, offsets, family, precision="f32c", weight="invvar", ctx: Optional[Context] = None, stream=None,
        opts: Optional[Opts] = None) -> FitResult:
    """Divide-and-combine MPL fit of one dataset on the GPU.

    u, v: CUDA tensors (float32 or float64) holding the two columns; offsets:
    K+1 host row offsets of the subsets (Eq. 14)."""
    torch = _torch()
    ctx = ctx or context()
    off = _offsets(offsets)
    K = off.shape[0] - 1
    dt = _dtype_code(u)
    if v.dtype != u.dtype or u.shape != v.shape or not u.is_cuda:
        raise CopulaError("u and v must be CUDA tensors of one dtype and shape")
    u = u.contiguous()
    v = v.contiguous()
    o = opts or make_opts(precision, weight)
    ws = ctx.workspace(ctx.workspace_size("copula_fit_workspace_size", dt, o, off), u.device)
    theta = torch.empty(K, dtype=torch.float64, device=u.device)
    var = torch.empty(K, dtype=torch.float64, device=u.device)
    status = torch.empty(K, dtype=torch.int32, device=u.device)
    comb = torch.empty(1, dtype=torch.float64, device=u.device)
    ctx.check(lib().copula_fit(ctx.handle, _family(family), dt, u.data_ptr(), v.data_ptr(), u.shape[0],
                               off.ctypes.data_as(_i64p), K, theta.data_ptr(), var.data_ptr(), status.data_ptr(),
                               comb.data_ptr(), ctypes.byref(o), ws.data_ptr(), ws.numel(), _stream(stream)),
              "copula_fit")
    return FitResult(theta, var, status, comb)


@dataclass
class FitDiagnostics:
    info: object       # [K] float64: observed information at theta_hat
    iters: object      # [K] int32: likelihood passes of the Newton driver
    phase_ns: object   # [K, 4] int64: global-timer stamps (start, ranked, searched, end)


def fit_ex(u, v, offsets, family, precision="f32c", weight="invvar", ctx: Optional[Context] = None, stream=None,
           opts: Optional[Opts] = None, phases: bool = False):
    """fit() plus per-subset diagnostics (copula_fit_ex)."""
    torch = _torch()
    ctx = ctx or context()
    off = _offsets(offsets)
    K = off.shape[0] - 1
    dt = _dtype_code(u)
    u = u.contiguous()
    v = v.contiguous()
    o = opts or make_opts(precision, weight)
    nb = _sz()
    ctx.check(lib().copula_fit_workspace_size(ctx.handle, dt, ctypes.byref(o), off.ctypes.data_as(_i64p), K,
                                              ctypes.byref(nb)), "copula_fit_workspace_size")
    ws = ctx.workspace(nb.value, u.device)
    dv = u.device
    theta, var = torch.empty(K, dtype=torch.float64, device=dv), torch.empty(K, dtype=torch.float64, device=dv)
    status, comb = torch.empty(K, dtype=torch.int32, device=dv), torch.empty(1, dtype=torch.float64, device=dv)
    info, iters = torch.empty(K, dtype=torch.float64, device=dv), torch.empty(K, dtype=torch.int32, device=dv)
    ph = torch.zeros((K, 4), dtype=torch.int64, device=dv) if phases else None
    ctx.check(lib().copula_fit_ex(ctx.handle, _family(family), dt, u.data_ptr(), v.data_ptr(), u.shape[0],
                                  off.ctypes.data_as(_i64p), K, theta.data_ptr(), var.data_ptr(), status.data_ptr(),
                                  comb.data_ptr(), info.data_ptr(), iters.data_ptr(),
                                  ph.data_ptr() if ph is not None else None, ctypes.byref(o), ws.data_ptr(),
                                  ws.numel(), _stream(stream)), "copula_fit_ex")
    return FitResult(theta, var, status, comb), FitDiagnostics(info, iters, ph)


def fit_batch(u, v, families: Sequence[int], dataset_offsets, subset_offsets, dataset_subset_start,
              precision="f32c", weight="invvar", ctx: Optional[Context] = None, stream=None,
              opts: Optional[Opts] = None) -> FitResult:
    """Batched fit of B datasets (concatenated in u, v) in one launch sequence."""
    torch = _torch()
    ctx = ctx or context()
    dofs, soff, dss = _offsets(dataset_offsets), _offsets(subset_offsets), _offsets(dataset_subset_start)
    fam = np.ascontiguousarray(np.asarray([_family(f) for f in families], dtype=np.int32))
    B = fam.shape[0]
    S = int(dss[-1])
    dt = _dtype_code(u)
    u = u.contiguous()
    v = v.contiguous()
    o = opts or make_opts(precision, weight)
    nb = _sz()
    ctx.check(lib().copula_fit_batch_workspace_size(ctx.handle, dt, ctypes.byref(o), B, fam.ctypes.data_as(_i32p),
                                                    dofs.ctypes.data_as(_i64p), soff.ctypes.data_as(_i64p),
                                                    dss.ctypes.data_as(_i64p), ctypes.byref(nb)),
              "copula_fit_batch_workspace_size")
    ws = ctx.workspace(nb.value, u.device)
    theta = torch.empty(S, dtype=torch.float64, device=u.device)
    var = torch.empty(S, dtype=torch.float64, device=u.device)
    status = torch.empty(S, dtype=torch.int32, device=u.device)
    comb = torch.empty(B, dtype=torch.float64, device=u.device)
    ctx.check(lib().copula_fit_batch(ctx.handle, B, fam.ctypes.data_as(_i32p), dt, u.data_ptr(), v.data_ptr(),
                                     dofs.ctypes.data_as(_i64p), soff.ctypes.data_as(_i64p),
                                     dss.ctypes.data_as(_i64p), theta.data_ptr(), var.data_ptr(), status.data_ptr(),
                                     comb.data_ptr(), ctypes.byref(o), ws.data_ptr(), ws.numel(), _stream(stream)),
              "copula_fit_batch")
    return FitResult(theta, var, status, comb)


def fit_host(u: np.ndarray, v: np.ndarray, offsets, family, precision="f32c", weight="invvar",
             ctx: Optional[Context] = None, stream=None, opts: Optional[Opts] = None, out=None):
    """copula_fit_host: host arrays in, host arrays out (copies inside the call).

    u, v: numpy arrays or pinned CPU torch tensors.  Returns numpy arrays
    (theta, var, status, combined)."""
    torch = _torch()
    ctx = ctx or context()
    off = _offsets(offsets)
    K = off.shape[0] - 1
    if isinstance(u, np.ndarray):
        up, vp_, dt, n = u.ctypes.data, v.ctypes.data, (DTYPE_F32 if u.dtype == np.float32 else DTYPE_F64), u.shape[0]
    else:
        up, vp_, dt, n = u.data_ptr(), v.data_ptr(), _dtype_code(u), u.shape[0]
    o = opts or make_opts(precision, weight)
    nb = ctx.workspace_size("copula_fit_host_workspace_size", dt, o, off)
    ws = ctx.workspace(nb, torch.device("cuda", torch.cuda.current_device()))
    if out is None:
        out = (np.empty(K), np.empty(K), np.empty(K, dtype=np.int32), np.empty(1))
    th, var, st, comb = out
    ctx.check(lib().copula_fit_host(ctx.handle, _family(family), dt, up, vp_, n, off.ctypes.data_as(_i64p), K,
                                    th.ctypes.data, var.ctypes.data, st.ctypes.data, comb.ctypes.data,
                                    ctypes.byref(o), ws.data_ptr(), ws.numel(), _stream(stream)), "copula_fit_host")
    return th, var, st, comb


def fit_batch_host(u, v, families: Sequence[int], dataset_offsets, subset_offsets, dataset_subset_start,
                   precision="f32c", weight="invvar", ctx: Optional[Context] = None, stream=None,
                   opts: Optional[Opts] = None, out=None):
    """copula_fit_batch_host: host columns of B datasets in, host results out.

    u, v: numpy arrays or (pinned) CPU torch tensors.  Returns numpy arrays
    (theta [S], var [S], status [S], combined [B])."""
    torch = _torch()
    ctx = ctx or context()
    dofs, soff, dss = _offsets(dataset_offsets), _offsets(subset_offsets), _offsets(dataset_subset_start)
    fam = np.ascontiguousarray(np.asarray([_family(f) for f in families], dtype=np.int32))
    B = fam.shape[0]
    S = int(dss[-1])
    if isinstance(u, np.ndarray):
        up, vp_, dt = u.ctypes.data, v.ctypes.data, (DTYPE_F32 if u.dtype == np.float32 else DTYPE_F64)
    else:
        up, vp_, dt = u.data_ptr(), v.data_ptr(), _dtype_code(u)
    o = opts or make_opts(precision, weight)
    nb = _sz()
    ctx.check(lib().copula_fit_batch_host_workspace_size(ctx.handle, dt, ctypes.byref(o), B,
                                                         fam.ctypes.data_as(_i32p),
                                                         dofs.ctypes.data_as(_i64p), soff.ctypes.data_as(_i64p),
                                                         dss.ctypes.data_as(_i64p), ctypes.byref(nb)),
              "copula_fit_batch_host_workspace_size")
    ws = ctx.workspace(nb.value, torch.device("cuda", torch.cuda.current_device()))
    if out is None:
        out = (np.empty(S), np.empty(S), np.empty(S, dtype=np.int32), np.empty(B))
    th, var, st, comb = out
    ctx.check(lib().copula_fit_batch_host(ctx.handle, B, fam.ctypes.data_as(_i32p), dt, up, vp_,
                                          dofs.ctypes.data_as(_i64p), soff.ctypes.data_as(_i64p),
                                          dss.ctypes.data_as(_i64p), th.ctypes.data, var.ctypes.data,
                                          st.ctypes.data, comb.ctypes.data, ctypes.byref(o), ws.data_ptr(),
                                          ws.numel(), _stream(stream)), "copula_fit_batch_host")
    return th, var, st, comb


UNIT_RATES = ("mufu_ex2", "mufu_lg2", "mufu_rcp", "fp32_fma", "fp64_fma")


def measure_unit_rates() -> dict:
    """copula_measure_unit_rates: measured results/s of the MUFU ex2, lg2 and
    rcp approximations and of FP32 and FP64 FMA on the current GPU."""
    _torch()
    out = (_d * len(UNIT_RATES))()
    rc = lib().copula_measure_unit_rates(out, len(UNIT_RATES), None)
    if rc != 0:
        raise CopulaError(f"copula_measure_unit_rates failed ({rc})")
    return {k: float(out[i]) for i, k in enumerate(UNIT_RATES)}


def ranks(x, offsets, ctx: Optional[Context] = None, stream=None):
    """Within-subset ordinal ranks 1..m of a CUDA column (Eq. 12)."""
    torch = _torch()
    ctx = ctx or context()
    off = _offsets(offsets)
    K = off.shape[0] - 1
    dt = _dtype_code(x)
    x = x.contiguous()
    o = make_opts()
    nb = _sz()
    ctx.check(lib().copula_fit_workspace_size(ctx.handle, dt, ctypes.byref(o), off.ctypes.data_as(_i64p), K,
                                              ctypes.byref(nb)), "copula_fit_workspace_size")
    ws = ctx.workspace(nb.value, x.device)
    out = torch.empty(x.shape[0], dtype=torch.int32, device=x.device)
    ctx.check(lib().copula_ranks(ctx.handle, dt, x.data_ptr(), x.shape[0], off.ctypes.data_as(_i64p), K,
                                 out.data_ptr(), ws.data_ptr(), ws.numel(), _stream(stream)), "copula_ranks")
    return out


def rank_corr(u, v, offsets, ctx: Optional[Context] = None, stream=None):
    """Kendall's tau and Spearman's rho of every subset's ranks (copula_rank_corr):
    two CUDA float64 tensors of K values."""
    torch = _torch()
    ctx = ctx or context()
    off = _offsets(offsets)
    K = off.shape[0] - 1
    dt = _dtype_code(u)
    if v.dtype != u.dtype or u.shape != v.shape or not u.is_cuda:
        raise CopulaError("u and v must be CUDA tensors of one dtype and shape")
    u = u.contiguous()
    v = v.contiguous()
    ws = ctx.workspace(ctx.workspace_size("copula_fit_workspace_size", dt, make_opts(), off), u.device)
    tau = torch.empty(K, dtype=torch.float64, device=u.device)
    rho = torch.empty(K, dtype=torch.float64, device=u.device)
    ctx.check(lib().copula_rank_corr(ctx.handle, dt, u.data_ptr(), v.data_ptr(), u.shape[0],
                                     off.ctypes.data_as(_i64p), K, tau.data_ptr(), rho.data_ptr(), ws.data_ptr(),
                                     ws.numel(), _stream(stream)), "copula_rank_corr")
    return tau, rho


def theta_from_rank_corr(r, family, which="tau", stream=None):
    """copula_theta_from_rank_corr: the parameter of `family` whose population
    Kendall's tau (which="tau") or Spearman's rho (which="rho") equals each
    value of the CUDA float64 tensor r.  Returns (theta, status) tensors."""
    torch = _torch()
    r = torch.as_tensor(r, dtype=torch.float64, device="cuda").contiguous()
    K = r.shape[0]
    theta = torch.empty(K, dtype=torch.float64, device=r.device)
    status = torch.empty(K, dtype=torch.int32, device=r.device)
    w = {"tau": 0, "rho": 1}[which] if isinstance(which, str) else int(which)
    rc = lib().copula_theta_from_rank_corr(_family(family), w, r.data_ptr(), K, theta.data_ptr(), status.data_ptr(),
                                           _stream(stream))
    if rc != 0:
        raise CopulaError(f"copula_theta_from_rank_corr failed ({rc})")
    return theta, status


def density_distance(family, theta_a, theta_b, delta: float = 0.0, stream=None):
    """copula_density_distance: for each pair (theta_a[k], theta_b[k]) the four
    integrals over [delta, 1-delta]^2 of |ca - cb|, |ca|, (ca - cb)^2, ca^2
    ([K, 4]) and the relative L1 / L2 distances of Eq. 19-20 ([K, 2])."""
    torch = _torch()
    ta = torch.as_tensor(theta_a, dtype=torch.float64, device="cuda").reshape(-1).contiguous()
    tb = torch.as_tensor(theta_b, dtype=torch.float64, device="cuda").reshape(-1).contiguous()
    K = ta.shape[0]
    nb = _sz()
    if lib().copula_density_distance_workspace_size(_family(family), float(delta), K, ctypes.byref(nb)) != 0:
        raise CopulaError("copula_density_distance_workspace_size: bad arguments")
    ws = torch.empty(max(nb.value, 256), dtype=torch.uint8, device="cuda")
    integ = torch.empty((K, 4), dtype=torch.float64, device="cuda")
    rel = torch.empty((K, 2), dtype=torch.float64, device="cuda")
    rc = lib().copula_density_distance(_family(family), float(delta), K, ta.data_ptr(), tb.data_ptr(),
                                       integ.data_ptr(), rel.data_ptr(), ws.data_ptr(), ws.numel(), _stream(stream))
    if rc != 0:
        raise CopulaError(f"copula_density_distance failed ({rc})")
    return integ, rel


SIM_SUMMARY = ("theta_combined_sim", "theta_full_sim", "bias", "mse", "d1_relative", "d2_relative",
               "int_abs_diff", "int_abs", "int_sq_diff", "int_sq")


def simulation_summary(family, theta_combined, theta_full, delta: float = 0.0, stream=None):
    """copula_simulation_summary: Eq. 17, Eq. 18, bias, MSE and Eq. 19-20 of S
    simulations from their combined and full-data estimates (CUDA float64
    tensors).  Returns a CUDA float64 tensor of 10 values (SIM_SUMMARY)."""
    torch = _torch()
    tc = torch.as_tensor(theta_combined, dtype=torch.float64, device="cuda").reshape(-1).contiguous()
    tf = torch.as_tensor(theta_full, dtype=torch.float64, device="cuda").reshape(-1).contiguous()
    if tc.shape != tf.shape:
        raise CopulaError("theta_combined and theta_full must have one length")
    nb = _sz()
    if lib().copula_simulation_summary_workspace_size(_family(family), float(delta), ctypes.byref(nb)) != 0:
        raise CopulaError("copula_simulation_summary_workspace_size: bad arguments")
    ws = torch.empty(max(nb.value, 256), dtype=torch.uint8, device="cuda")
    out = torch.empty(len(SIM_SUMMARY), dtype=torch.float64, device="cuda")
    rc = lib().copula_simulation_summary(_family(family), float(delta), tc.shape[0], tc.data_ptr(), tf.data_ptr(),
                                         out.data_ptr(), ws.data_ptr(), ws.numel(), _stream(stream))
    if rc != 0:
        raise CopulaError(f"copula_simulation_summary failed ({rc})")
    return out


def loglik(u, v, offsets, family, theta, precision="f32c", ctx: Optional[Context] = None, stream=None):
    """One likelihood pass: (sum l, sum dl/dtheta, sum d2l/dtheta2) per subset
    at the given per-subset parameters (Eq. 13)."""
    torch = _torch()
    ctx = ctx or context()
    off = _offsets(offsets)
    K = off.shape[0] - 1
    dt = _dtype_code(u)
    theta = torch.as_tensor(theta, dtype=torch.float64, device=u.device).contiguous()
    o = make_opts(precision)
    nb = _sz()
    ctx.check(lib().copula_fit_workspace_size(ctx.handle, dt, ctypes.byref(o), off.ctypes.data_as(_i64p), K,
                                              ctypes.byref(nb)), "copula_fit_workspace_size")
    ws = ctx.workspace(nb.value, u.device)
    l, g, h = (torch.empty(K, dtype=torch.float64, device=u.device) for _ in range(3))
    ctx.check(lib().copula_loglik(ctx.handle, _family(family), dt, u.contiguous().data_ptr(),
                                  v.contiguous().data_ptr(), u.shape[0], off.ctypes.data_as(_i64p), K,
                                  theta.data_ptr(), l.data_ptr(), g.data_ptr(), h.data_ptr(), ctypes.byref(o),
                                  ws.data_ptr(), ws.numel(), _stream(stream)), "copula_loglik")
    return l, g, h


# ---------------------------------------------------------------------------
# Serving (copula_server_*) and its arena allocator (copula_arena_*).
# ---------------------------------------------------------------------------

class _CRequest(ctypes.Structure):
    _fields_ = [("family", _i32), ("dtype", _i32), ("u", _vp), ("v", _vp), ("n", _i64), ("subset_offsets", _i64p),
                ("K", _i64), ("opts", Opts), ("theta_out", _vp), ("var_out", _vp), ("status_out", _vp)]


class _CResult(ctypes.Structure):
    _fields_ = [("state", _i32), ("rc", _i32), ("theta_combined", _d), ("latency_s", _d), ("queue_s", _d)]


class _CStats(ctypes.Structure):
    _fields_ = [("fits_done", _i64), ("errors", _i64), ("batches", _i64), ("pending", _i64), ("mean_batch", _d),
                ("max_inflight_batches", _i32), ("reserved", _i32), ("fits_per_s", _d), ("p50_s", _d), ("p99_s", _d),
                ("mean_queue_s", _d), ("arena_peak_bytes", _sz)]


REQ_PENDING, REQ_RUNNING, REQ_DONE, REQ_ERROR = 0, 1, 2, 3
_serve_ready = False


def _serve_lib():
    global _serve_ready
    L = lib()
    if not _serve_ready:
        L.copula_arena_create.argtypes = [ctypes.POINTER(_vp), _sz]
        L.copula_arena_destroy.argtypes = [_vp]
        L.copula_arena_alloc.argtypes = [_vp, _sz, ctypes.POINTER(_sz)]
        L.copula_arena_free.argtypes = [_vp, _sz]
        L.copula_arena_stats.argtypes = [_vp, ctypes.POINTER(_sz), ctypes.POINTER(_sz), ctypes.POINTER(_sz)]
        L.copula_server_create.argtypes = [ctypes.POINTER(_vp), _vp, _sz, _i32, _i32]
        L.copula_server_submit.argtypes = [_vp, ctypes.POINTER(_CRequest), ctypes.POINTER(ctypes.c_uint64)]
        L.copula_server_poll.argtypes = [_vp, ctypes.c_uint64, ctypes.POINTER(_CResult)]
        L.copula_server_wait.argtypes = [_vp, ctypes.c_uint64, _d, ctypes.POINTER(_CResult)]
        L.copula_server_stats.argtypes = [_vp, ctypes.POINTER(_CStats)]
        L.copula_server_reset_stats.argtypes = [_vp]
        L.copula_server_destroy.argtypes = [_vp]
        _serve_ready = True
    return L


class Arena:
    """First-fit offset allocator of the serving loop (host bookkeeping only)."""

    def __init__(self, nbytes: int):
        self._h = _vp()
        if _serve_lib().copula_arena_create(ctypes.byref(self._h), int(nbytes)) != 0:
            raise CopulaError("copula_arena_create failed")

    def alloc(self, nbytes: int):
        off = _sz()
        rc = _serve_lib().copula_arena_alloc(self._h, int(nbytes), ctypes.byref(off))
        return off.value if rc == 0 else None

    def free(self, off: int) -> bool:
        return _serve_lib().copula_arena_free(self._h, int(off)) == 0

    def stats(self):
        u, p, b = _sz(), _sz(), _sz()
        _serve_lib().copula_arena_stats(self._h, ctypes.byref(u), ctypes.byref(p), ctypes.byref(b))
        return {"used": u.value, "peak": p.value, "largest_free": b.value}

    def close(self):
        if self._h:
            _serve_lib().copula_arena_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching fit server (copula_server_*) on the current device.

    budget_bytes of device memory is taken once (a torch tensor) and handed
    to the server as its arena; requests are numpy arrays kept alive here
    until they complete."""

    def __init__(self, budget_bytes: int, max_slots: int = 64, streams: int = 4):
        torch = _torch()
        self._arena = torch.empty(int(budget_bytes), dtype=torch.uint8, device="cuda")
        self._h = _vp()
        rc = _serve_lib().copula_server_create(ctypes.byref(self._h), self._arena.data_ptr(), int(budget_bytes),
                                               int(max_slots), int(streams))
        if rc != 0:
            raise CopulaError(f"copula_server_create failed ({rc})")
        self._live = {}

    def submit(self, u: np.ndarray, v: np.ndarray, offsets, family, precision="f32c", weight="invvar",
               opts: Optional[Opts] = None) -> int:
        u = np.ascontiguousarray(u)
        v = np.ascontiguousarray(v)
        off = _offsets(offsets)
        K = off.shape[0] - 1
        th, var, st = np.empty(K), np.empty(K), np.empty(K, dtype=np.int32)
        r = _CRequest()
        r.family = _family(family)
        r.dtype = DTYPE_F32 if u.dtype == np.float32 else DTYPE_F64
        r.u, r.v, r.n = u.ctypes.data, v.ctypes.data, u.shape[0]
        r.subset_offsets = off.ctypes.data_as(_i64p)
        r.K = K
        r.opts = opts or make_opts(precision, weight)
        r.theta_out, r.var_out, r.status_out = th.ctypes.data, var.ctypes.data, st.ctypes.data
        t = ctypes.c_uint64()
        rc = _serve_lib().copula_server_submit(self._h, ctypes.byref(r), ctypes.byref(t))
        if rc != 0:
            raise CopulaError(f"copula_server_submit failed ({rc})")
        self._live[t.value] = (u, v, th, var, st)
        return t.value

    def _result(self, ticket, res):
        out = {"state": res.state, "rc": res.rc, "combined": res.theta_combined, "latency_s": res.latency_s,
               "queue_s": res.queue_s}
        if res.state in (REQ_DONE, REQ_ERROR):
            u, v, th, var, st = self._live.pop(ticket)
            out.update(theta=th, var=var, status=st)
        return out

    def poll(self, ticket: int):
        res = _CResult()
        if _serve_lib().copula_server_poll(self._h, ticket, ctypes.byref(res)) != 0:
            raise CopulaError("unknown ticket")
        return self._result(ticket, res)

    def wait(self, ticket: int, timeout_s: float = 0.0):
        res = _CResult()
        if _serve_lib().copula_server_wait(self._h, ticket, float(timeout_s), ctypes.byref(res)) != 0:
            raise CopulaError("unknown ticket")
        return self._result(ticket, res)

    def stats(self):
        s = _CStats()
        _serve_lib().copula_server_stats(self._h, ctypes.byref(s))
        return {f: getattr(s, f) for f, _ in _CStats._fields_ if f != "reserved"}

    def reset_stats(self):
        _serve_lib().copula_server_reset_stats(self._h)

    def close(self):
        if self._h:
            _serve_lib().copula_server_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Plans (copula_plan_*): a batched fit whose launches can be captured into a
# CUDA graph, and the per-context block-size table (copula_ctx_set_blocks).
# ---------------------------------------------------------------------------

_plan_ready = False


def _plan_lib():
    global _plan_ready
    L = lib()
    if not _plan_ready:
        L.copula_plan_create.argtypes = [_vp, ctypes.POINTER(_vp), _i32, _i32p, _i32, _i64p, _i64p, _i64p,
                                         ctypes.POINTER(Opts), ctypes.POINTER(_sz)]
        L.copula_plan_upload.argtypes = [_vp, _vp, _sz, _vp]
        L.copula_plan_run.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]
        L.copula_plan_destroy.argtypes = [_vp]
        L.copula_plan_diagnostics.argtypes = [_vp, _vp, _sz, _vp, _vp, _vp]
        L.copula_ctx_set_blocks.argtypes = [_vp, _i32p, _i32p, _i32]
        L.copula_ctx_set_family_blocks.argtypes = [_vp, _i32, _i32p, _i32p, _i32]
        _plan_ready = True
    return L


def set_blocks(table, ctx: Optional[Context] = None, family=None):
    """Per-size block table: list of (largest m, threads), increasing m; for
    every family, or for one (copula_ctx_set_family_blocks)."""
    ctx = ctx or context()
    mm = np.ascontiguousarray([t[0] for t in table], dtype=np.int32)
    th = np.ascontiguousarray([t[1] for t in table], dtype=np.int32)
    if family is None:
        ctx.check(_plan_lib().copula_ctx_set_blocks(ctx.handle, mm.ctypes.data_as(_i32p), th.ctypes.data_as(_i32p),
                                                    len(table)), "copula_ctx_set_blocks")
    else:
        ctx.check(_plan_lib().copula_ctx_set_family_blocks(ctx.handle, _family(family), mm.ctypes.data_as(_i32p),
                                                           th.ctypes.data_as(_i32p), len(table)),
                  "copula_ctx_set_family_blocks")
    ctx._sizes.clear()  # block sizes change the plans, so the workspace sizes


class BatchPlan:
    """A fixed batch of datasets (families and partitions) fitted by one
    launch sequence that only touches device memory; `capture()` records it
    as a CUDA graph that can be replayed on new data in the same buffers."""

    def __init__(self, families, dataset_offsets, subset_offsets, dataset_subset_start, dtype="f32",
                 precision="f32c", weight="invvar", ctx: Optional[Context] = None, opts: Optional[Opts] = None):
        torch = _torch()
        self.ctx = ctx or context()
        self._fam = np.ascontiguousarray(np.asarray([_family(f) for f in families], dtype=np.int32))
        self._dofs = _offsets(dataset_offsets)
        self._soff = _offsets(subset_offsets)
        self._dss = _offsets(dataset_subset_start)
        self.B = self._fam.shape[0]
        self.S = int(self._dss[-1])
        self.n = int(self._dofs[-1])
        self.dtype = DTYPE_F32 if dtype in ("f32", np.float32) else DTYPE_F64
        o = opts or make_opts(precision, weight)
        self._h = _vp()
        nb = _sz()
        self.ctx.check(_plan_lib().copula_plan_create(self.ctx.handle, ctypes.byref(self._h), self.B,
                                                      self._fam.ctypes.data_as(_i32p), self.dtype,
                                                      self._dofs.ctypes.data_as(_i64p),
                                                      self._soff.ctypes.data_as(_i64p),
                                                      self._dss.ctypes.data_as(_i64p), ctypes.byref(o),
                                                      ctypes.byref(nb)), "copula_plan_create")
        self.workspace = torch.empty(max(nb.value, 256), dtype=torch.uint8, device="cuda")
        self.ctx.check(_plan_lib().copula_plan_upload(self._h, self.workspace.data_ptr(), self.workspace.numel(),
                                                      _stream(None)), "copula_plan_upload")
        dv = torch.device("cuda", torch.cuda.current_device())
        self.theta = torch.empty(self.S, dtype=torch.float64, device=dv)
        self.var = torch.empty(self.S, dtype=torch.float64, device=dv)
        self.status = torch.empty(self.S, dtype=torch.int32, device=dv)
        self.combined = torch.empty(self.B, dtype=torch.float64, device=dv)

    def run(self, u, v, stream=None):
        """Enqueue one fit of the batch held in u, v (CUDA, n values each)."""
        assert u.is_cuda and v.is_cuda and u.shape[0] == self.n and u.is_contiguous() and v.is_contiguous()
        self.ctx.check(_plan_lib().copula_plan_run(self._h, u.data_ptr(), v.data_ptr(), self.theta.data_ptr(),
                                                   self.var.data_ptr(), self.status.data_ptr(),
                                                   self.combined.data_ptr(), self.workspace.data_ptr(),
                                                   self.workspace.numel(), _stream(stream)), "copula_plan_run")
        return FitResult(self.theta, self.var, self.status, self.combined)

    def diagnostics(self, stream=None):
        """(info [S], iters [S]) of the last run: observed information and
        Newton passes per subset (copula_plan_diagnostics)."""
        torch = _torch()
        info = torch.empty(self.S, dtype=torch.float64, device=self.theta.device)
        iters = torch.empty(self.S, dtype=torch.int32, device=self.theta.device)
        self.ctx.check(_plan_lib().copula_plan_diagnostics(self._h, self.workspace.data_ptr(),
                                                           self.workspace.numel(), info.data_ptr(),
                                                           iters.data_ptr(), _stream(stream)),
                       "copula_plan_diagnostics")
        return info, iters

    def capture(self, u, v):
        """Record run(u, v) as a CUDA graph (after one warm-up run)."""
        torch = _torch()
        self.run(u, v)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run(u, v)
        return g

    def close(self):
        if self._h:
            _plan_lib().copula_plan_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
