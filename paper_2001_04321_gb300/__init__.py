"""GB300-native HER-accelerated block-coordinate descent for dense nonnegative
CP factorization (arXiv 2001.04321).

Thin Python binding over the C ABI of ``libntf.so`` (declared in
``include/ntf.h``).  This module only marshals arguments: torch CUDA tensors
become device pointers, the current torch stream becomes the ``stream``
argument, and every computation runs in the library's CUDA kernels.  There is
no CPU fallback: if ``libntf.so`` is missing or no CUDA device is present,
calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import List, Optional, Sequence

__all__ = [
    "NTFError", "lib", "load", "Opts", "Report", "mttkrp", "mttkrp_workspace_bytes", "gram",
    "hadamard_grams", "bcd_update", "her_extrapolate", "block_gradient", "CPLoss", "cp_loss", "objective", "residual_sq", "tensor_norm_sq",
    "to_bf16", "her_state_init", "her_step", "solve", "solve_host", "Solver", "launch_count",
    "device_status", "HER_STATE_BYTES", "Tucker", "tucker_mttkrp", "tucker_norm_sq", "solve_tucker",
    "mttkrp_streamed", "solve_streamed",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libntf.so")

NTF_F32, NTF_BF16 = 0, 1
NTF_HALS, NTF_PGD, NTF_NESTEROV = 0, 1, 2
_METHODS = {"hals": NTF_HALS, "pgd": NTF_PGD, "nesterov": NTF_NESTEROV}
_STATUS = {0: "NTF_OK", 1: "NTF_EINVAL", 2: "NTF_ENOMEM", 3: "NTF_ECUDA", 4: "NTF_ENUMERIC",
           5: "NTF_ETIMEOUT", 6: "NTF_ENOTSUP"}


class NTFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class _Tensor(C.Structure):
    _fields_ = [("order", C.c_int), ("dims", C.c_int64 * 8), ("dtype", C.c_int), ("ld", C.c_int64),
                ("data", C.c_void_p)]


class _Opts(C.Structure):
    _fields_ = [("her", C.c_int), ("method", C.c_int), ("inner_max", C.c_int), ("inner_tol", C.c_double),
                ("max_iters", C.c_int), ("beta0", C.c_double), ("gamma", C.c_double), ("gamma_bar", C.c_double),
                ("eta", C.c_double), ("compute_dtype", C.c_int), ("report_every", C.c_int), ("use_graph", C.c_int),
                ("max_seconds", C.c_double), ("rel_tol", C.c_double), ("check_every", C.c_int)]


class _Report(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("f_hat_last", C.c_double),
                ("f_true_last", C.c_double), ("rel_error", C.c_double), ("tnorm_sq", C.c_double),
                ("beta_last", C.c_double), ("beta_bar_last", C.c_double), ("seconds", C.c_double)]


class _Tucker(C.Structure):
    _fields_ = [("core", _Tensor), ("dims", C.c_int64 * 8), ("U", C.c_void_p * 8)]


class _HerState(C.Structure):
    _fields_ = [("beta", C.c_double), ("beta_bar", C.c_double), ("f_hat_prev", C.c_double),
                ("gamma", C.c_double), ("gamma_bar", C.c_double), ("eta", C.c_double), ("iters", C.c_int32),
                ("restarts", C.c_int32), ("last_restart", C.c_int32), ("numeric_error", C.c_int32)]


HER_STATE_BYTES = C.sizeof(_HerState)

_lib = None

# every exported symbol with its (restype, argtypes)
_P = C.c_void_p
_SIGS = {
    "ntf_last_error": (C.c_char_p, []),
    "ntf_device_status": (C.c_int, [_P]),
    "ntf_launch_count": (C.c_int64, []),
    "ntf_opts_default": (None, [C.POINTER(_Opts)]),
    "ntf_bf16_ld": (C.c_int64, [C.POINTER(_Tensor)]),
    "ntf_tensor_to_bf16": (C.c_int, [C.POINTER(_Tensor), _P, C.c_int64, _P]),
    "ntf_norm_workspace_bytes": (C.c_size_t, []),
    "ntf_tensor_norm_sq": (C.c_int, [C.POINTER(_Tensor), _P, _P, C.c_size_t, _P]),
    "ntf_mttkrp_workspace_bytes": (C.c_size_t, [C.POINTER(_Tensor), C.c_int, C.c_int]),
    "ntf_mttkrp": (C.c_int, [C.POINTER(_Tensor), C.POINTER(_P), C.c_int, C.c_int, _P, _P, C.c_size_t, _P]),
    "ntf_mttkrp_noalloc": (C.c_int, [C.POINTER(_Tensor), C.POINTER(_P), C.c_int, C.c_int, _P, _P]),
    "ntf_gram": (C.c_int, [_P, C.c_int64, C.c_int, _P, _P]),
    "ntf_hadamard_grams": (C.c_int, [C.POINTER(_P), C.c_int, C.c_int, C.c_int, _P, _P]),
    "ntf_bcd_workspace_bytes": (C.c_size_t, [C.c_int64, C.c_int]),
    "ntf_bcd_update": (C.c_int, [C.c_int, _P, C.c_int64, C.c_int, _P, _P, C.c_int, C.c_double, _P, C.c_size_t,
                                 _P]),
    "ntf_her_extrapolate": (C.c_int, [_P, _P, _P, C.c_int64, _P, _P]),
    "ntf_block_gradient": (C.c_int, [_P, C.c_int64, C.c_int, _P, _P, _P, C.c_double, _P, _P]),
    "ntf_check_wait_timeout": (C.c_int, [C.c_int64, _P]),
    "ntf_objective": (C.c_int, [_P, _P, _P, C.c_int64, C.c_int, _P, _P, _P]),
    "ntf_residual_workspace_bytes": (C.c_size_t, [C.POINTER(_Tensor), C.c_int]),
    "ntf_residual_sq": (C.c_int, [C.POINTER(_Tensor), C.POINTER(_P), C.c_int, _P, _P, C.c_size_t, _P]),
    "ntf_her_state_init": (C.c_int, [_P, C.c_double, C.c_double, C.c_double, C.c_double, _P, _P]),
    "ntf_her_step": (C.c_int, [_P, C.POINTER(_P), C.POINTER(_P), C.c_int, C.POINTER(C.c_int64), C.c_int, _P,
                               _P]),
    "ntf_solve": (C.c_int, [C.POINTER(_Tensor), C.POINTER(_P), C.c_int, C.POINTER(_Opts), C.POINTER(_Report),
                            _P]),
    "ntf_solve_host": (C.c_int, [C.POINTER(_Tensor), C.POINTER(_P), C.c_int, C.POINTER(_Opts),
                                 C.POINTER(_Report), _P]),
    "ntf_solver_create": (C.c_int, [C.POINTER(_P), C.POINTER(_Tensor), C.POINTER(_P), C.c_int, C.POINTER(_Opts),
                                    _P]),
    "ntf_solver_run": (C.c_int, [_P, C.c_int, _P]),
    "ntf_solver_prepare_graph": (C.c_int, [_P, C.c_int, _P]),
    "ntf_solver_get_factors": (C.c_int, [_P, C.POINTER(_P), _P]),
    "ntf_solver_report": (C.c_int, [_P, C.POINTER(_Report), _P]),
    "ntf_solver_set_timing": (C.c_int, [_P, C.c_int]),
    "ntf_solver_mttkrp_time": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                         C.POINTER(C.c_double), _P]),
    "ntf_solver_destroy": (None, [_P]),
    "ntf_tucker_mttkrp_workspace_bytes": (C.c_size_t, [C.POINTER(_Tucker), C.c_int, C.c_int]),
    "ntf_tucker_mttkrp": (C.c_int, [C.POINTER(_Tucker), C.POINTER(_P), C.c_int, C.c_int, _P, _P, C.c_size_t, _P]),
    "ntf_tucker_norm_workspace_bytes": (C.c_size_t, [C.POINTER(_Tucker)]),
    "ntf_tucker_norm_sq": (C.c_int, [C.POINTER(_Tucker), _P, _P, C.c_size_t, _P]),
    "ntf_mttkrp_streamed_workspace_bytes": (C.c_size_t, [C.POINTER(_Tensor), C.c_int, C.c_int, C.c_int64]),
    "ntf_mttkrp_streamed": (C.c_int, [C.POINTER(_Tensor), C.POINTER(_P), C.c_int, C.c_int, _P, _P, C.c_size_t,
                                      C.c_int64, _P]),
    "ntf_solve_tucker": (C.c_int, [C.POINTER(_Tucker), C.POINTER(_P), C.c_int, C.POINTER(_Opts), C.POINTER(_Report),
                                   _P]),
    "ntf_solve_streamed": (C.c_int, [C.POINTER(_Tensor), C.POINTER(_P), C.c_int, C.POINTER(_Opts),
                                     C.POINTER(_Report), C.c_int64, _P]),
    "ntf_solver_create_tucker": (C.c_int, [C.POINTER(_P), C.POINTER(_Tucker), C.POINTER(_P), C.c_int,
                                           C.POINTER(_Opts), _P]),
    "ntf_solver_create_streamed": (C.c_int, [C.POINTER(_P), C.POINTER(_Tensor), C.POINTER(_P), C.c_int,
                                             C.POINTER(_Opts), C.c_int64, _P]),
}
EXPORTED = tuple(_SIGS)


def load(path: str = LIB_PATH):
    """Load libntf.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise NTFError(6, f"{path} not found: build it with paper_2001_04321_gb300/build.py "
                              "(or __graft_entry__.build()); there is no CPU fallback")
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def lib():
    return load()


def _check(status: int):
    if status != 0:
        raise NTFError(status, load().ntf_last_error().decode(errors="replace"))


# ----------------------------------------------------------------------------
# marshalling helpers (torch is used only for device memory and streams)
# ----------------------------------------------------------------------------
def _torch():
    import torch
    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t) -> C.c_void_p:
    return C.c_void_p(t.data_ptr())


def _require_cuda(t, name: str, dtype=None, contiguous=True):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise NTFError(1, f"{name} must be a CUDA tensor (no CPU fallback)")
    if dtype is not None and t.dtype != dtype:
        raise NTFError(1, f"{name} must be {dtype}, got {t.dtype}")
    if contiguous and not t.is_contiguous():
        raise NTFError(1, f"{name} must be contiguous")


def _tensor_desc(T, dims: Optional[Sequence[int]] = None, ld: int = 0) -> _Tensor:
    """Describe a CUDA tensor: dense C-order (ld = 0) or, with ``dims`` and ``ld``,
    a row-padded buffer whose last-mode rows have pitch ``ld``."""
    torch = _torch()
    d = _Tensor()
    if dims is None:
        _require_cuda(T, "T")
        dims = list(T.shape)
    else:
        _require_cuda(T, "T")
    if T.dtype == torch.float32:
        d.dtype = NTF_F32
    elif T.dtype == torch.bfloat16:
        d.dtype = NTF_BF16
    else:
        raise NTFError(1, f"tensor dtype must be float32 or bfloat16, got {T.dtype}")
    d.order = len(dims)
    for i, v in enumerate(dims):
        d.dims[i] = int(v)
    d.ld = int(ld)
    d.data = T.data_ptr()
    return d


def _ptr_array(ts) -> "C.Array":
    arr = (_P * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = None if t is None else t.data_ptr()
    return arr


def check_wait_timeout(limit_ns: int = 10_000_000, stream=None) -> int:
    """Run the bounded-wait self-check; returns the status (NTF_ETIMEOUT when the path works)."""
    return int(load().ntf_check_wait_timeout(int(limit_ns), _stream(stream)))


def launch_count() -> int:
    return int(load().ntf_launch_count())


def device_status(stream=None):
    _check(load().ntf_device_status(_stream(stream)))


# ----------------------------------------------------------------------------
# single steps
# ----------------------------------------------------------------------------
def mttkrp_workspace_bytes(T, rank: int, mode: int, dims=None, ld: int = 0) -> int:
    d = _tensor_desc(T, dims, ld)
    return int(load().ntf_mttkrp_workspace_bytes(C.byref(d), rank, mode))


def mttkrp(T, factors: Sequence, mode: int, out=None, workspace=None, dims=None, ld: int = 0, stream=None):
    """MTTKRP of ``mode`` (0-based): ``out[j,p] = sum_{i_mode=j} T[i] prod_{l != mode} A_l[i_l, p]``."""
    torch = _torch()
    d = _tensor_desc(T, dims, ld)
    rank = int(factors[0 if mode != 0 else 1].shape[1])
    for l, A in enumerate(factors):
        if l != mode:
            _require_cuda(A, f"factor {l}", torch.float32)
    In = int(d.dims[mode])
    if out is None:
        out = torch.empty((In, rank), dtype=torch.float32, device=T.device)
    _require_cuda(out, "out", torch.float32)
    need = int(load().ntf_mttkrp_workspace_bytes(C.byref(d), rank, mode))
    if workspace is None:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=T.device)
    ptrs = _ptr_array([None if l == mode else A for l, A in enumerate(factors)])
    _check(load().ntf_mttkrp(C.byref(d), ptrs, rank, mode, _ptr(out), _ptr(workspace), workspace.numel(),
                             _stream(stream)))
    return out


def gram(A, out=None, stream=None):
    torch = _torch()
    _require_cuda(A, "A", torch.float32)
    r = int(A.shape[1])
    if out is None:
        out = torch.empty((r, r), dtype=torch.float64, device=A.device)
    _check(load().ntf_gram(_ptr(A), int(A.shape[0]), r, _ptr(out), _stream(stream)))
    return out


def hadamard_grams(grams: Sequence, skip: int, out=None, stream=None):
    torch = _torch()
    r = int(grams[0 if skip != 0 else 1].shape[0])
    if out is None:
        out = torch.empty((r, r), dtype=torch.float64, device=grams[0 if skip != 0 else 1].device)
    ptrs = _ptr_array([None if l == skip else g for l, g in enumerate(grams)])
    _check(load().ntf_hadamard_grams(ptrs, len(grams), skip, r, _ptr(out), _stream(stream)))
    return out


def bcd_update(A, M, V, method: str = "hals", inner_max: int = 1, inner_tol: float = 1e-2, workspace=None,
               stream=None):
    """In-place block update of ``A``: "hals", "pgd" or "nesterov" (AO-Nesterov)."""
    torch = _torch()
    _require_cuda(A, "A", torch.float32)
    _require_cuda(M, "M", torch.float32)
    _require_cuda(V, "V", torch.float64)
    rows, r = int(A.shape[0]), int(A.shape[1])
    need = int(load().ntf_bcd_workspace_bytes(rows, r))
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=A.device)
    m = _METHODS[method]
    _check(load().ntf_bcd_update(m, _ptr(A), rows, r, _ptr(M), _ptr(V), inner_max, inner_tol, _ptr(workspace),
                                 workspace.numel(), _stream(stream)))
    return A


def block_gradient(A, M, V, scale: float = 1.0, scale_dev=None, out=None, stream=None):
    """``scale * (A V - M)``: gradient of (1/2)||T - X||^2 with respect to ``A``."""
    torch = _torch()
    _require_cuda(A, "A", torch.float32)
    _require_cuda(M, "M", torch.float32)
    _require_cuda(V, "V", torch.float64)
    if out is None:
        out = torch.empty_like(A)
    _check(load().ntf_block_gradient(_ptr(A), int(A.shape[0]), int(A.shape[1]), _ptr(M), _ptr(V),
                                     None if scale_dev is None else _ptr(scale_dev), float(scale), _ptr(out),
                                     _stream(stream)))
    return out


def her_extrapolate(A, A_prev, beta_dev, out=None, stream=None):
    torch = _torch()
    if out is None:
        out = torch.empty_like(A)
    _check(load().ntf_her_extrapolate(_ptr(A), _ptr(A_prev), _ptr(beta_dev), A.numel(), _ptr(out),
                                      _stream(stream)))
    return out


def objective(tnorm_sq_dev, M, A, V, out=None, stream=None):
    torch = _torch()
    if out is None:
        out = torch.empty((), dtype=torch.float64, device=A.device)
    _check(load().ntf_objective(_ptr(tnorm_sq_dev), _ptr(M), _ptr(A), int(A.shape[0]), int(A.shape[1]), _ptr(V),
                                _ptr(out), _stream(stream)))
    return out


def tensor_norm_sq(T, out=None, dims=None, ld: int = 0, stream=None):
    torch = _torch()
    d = _tensor_desc(T, dims, ld)
    if out is None:
        out = torch.empty((), dtype=torch.float64, device=T.device)
    ws = torch.empty(int(load().ntf_norm_workspace_bytes()), dtype=torch.uint8, device=T.device)
    _check(load().ntf_tensor_norm_sq(C.byref(d), _ptr(out), _ptr(ws), ws.numel(), _stream(stream)))
    return out


def residual_sq(T, factors: Sequence, out=None, dims=None, ld: int = 0, stream=None):
    torch = _torch()
    d = _tensor_desc(T, dims, ld)
    rank = int(factors[0].shape[1])
    if out is None:
        out = torch.empty((), dtype=torch.float64, device=T.device)
    need = int(load().ntf_residual_workspace_bytes(C.byref(d), rank))
    ws = torch.empty(need, dtype=torch.uint8, device=T.device)
    _check(load().ntf_residual_sq(C.byref(d), _ptr_array(factors), rank, _ptr(out), _ptr(ws), ws.numel(),
                                  _stream(stream)))
    return out


def to_bf16(T, stream=None):
    """bfloat16 copy (round to nearest even) with 16-byte rows; returns (buffer, dims, ld)."""
    torch = _torch()
    d = _tensor_desc(T)
    ld = int(load().ntf_bf16_ld(C.byref(d)))
    rows = 1
    for v in T.shape[:-1]:
        rows *= int(v)
    buf = torch.empty(rows * ld, dtype=torch.bfloat16, device=T.device)
    _check(load().ntf_tensor_to_bf16(C.byref(d), _ptr(buf), ld, _stream(stream)))
    return buf, list(T.shape), ld


def her_state_init(state_buf, f_hat0_dev, beta0=0.5, gamma=1.05, gamma_bar=1.01, eta=1.5, stream=None):
    _check(load().ntf_her_state_init(_ptr(state_buf), beta0, gamma, gamma_bar, eta, _ptr(f_hat0_dev),
                                     _stream(stream)))


def her_step(state_buf, A: Sequence, A_hat: Sequence, f_hat_dev, stream=None):
    rows = (C.c_int64 * len(A))(*[int(a.shape[0]) for a in A])
    _check(load().ntf_her_step(_ptr(state_buf), _ptr_array(A), _ptr_array(A_hat), len(A), rows,
                               int(A[0].shape[1]), _ptr(f_hat_dev), _stream(stream)))


def her_state_read(state_buf) -> dict:
    raw = state_buf.cpu().numpy().tobytes()
    s = _HerState.from_buffer_copy(raw[:C.sizeof(_HerState)])
    return {f: getattr(s, f) for f, _ in _HerState._fields_}


# ----------------------------------------------------------------------------
# solver
# ----------------------------------------------------------------------------
@dataclass
class Opts:
    her: bool = True
    method: str = "hals"
    inner_max: int = 1
    inner_tol: float = 1e-2
    max_iters: int = 100
    beta0: float = 0.5
    gamma: float = 1.05
    gamma_bar: float = 1.01
    eta: float = 1.5
    compute_dtype: str = "f32"
    report_every: int = 0
    use_graph: bool = False
    max_seconds: float = 0.0
    rel_tol: float = 0.0
    check_every: int = 0

    def c(self) -> _Opts:
        o = _Opts()
        load().ntf_opts_default(C.byref(o))
        o.her = int(self.her)
        o.method = _METHODS[self.method]
        o.inner_max = int(self.inner_max)
        o.inner_tol = float(self.inner_tol)
        o.max_iters = int(self.max_iters)
        o.beta0, o.gamma, o.gamma_bar, o.eta = self.beta0, self.gamma, self.gamma_bar, self.eta
        o.compute_dtype = NTF_BF16 if self.compute_dtype == "bf16" else NTF_F32
        o.report_every = int(self.report_every)
        o.use_graph = int(self.use_graph)
        o.max_seconds = float(self.max_seconds)
        o.rel_tol = float(self.rel_tol)
        o.check_every = int(self.check_every)
        return o


@dataclass
class Report:
    iters: int
    restarts: int
    f_hat_last: float
    f_true_last: float
    rel_error: float
    tnorm_sq: float
    beta_last: float
    beta_bar_last: float
    seconds: float


def _report(r: _Report) -> Report:
    return Report(*(getattr(r, f) for f, _ in _Report._fields_))


def solve(T, factors: List, opts: Optional[Opts] = None, dims=None, ld: int = 0, stream=None) -> Report:
    """Run Alg. 2 (or Alg. 1) in place on the CUDA ``factors`` (list of (I_l, r) float32)."""
    torch = _torch()
    d = _tensor_desc(T, dims, ld)
    for A in factors:
        _require_cuda(A, "factor", torch.float32)
    o = (opts or Opts()).c()
    rep = _Report()
    _check(load().ntf_solve(C.byref(d), _ptr_array(factors), int(factors[0].shape[1]), C.byref(o), C.byref(rep),
                            _stream(stream)))
    return _report(rep)


def solve_host(T_host, factors_host: List, opts: Optional[Opts] = None, stream=None) -> Report:
    """``ntf_solve_host``: T and factors are host torch tensors (pin them for full copy speed)."""
    torch = _torch()
    d = _Tensor()
    if T_host.dtype != torch.float32 or T_host.is_cuda or not T_host.is_contiguous():
        raise NTFError(1, "T_host must be a contiguous host float32 tensor")
    d.order = T_host.dim()
    for i, v in enumerate(T_host.shape):
        d.dims[i] = int(v)
    d.dtype = NTF_F32
    d.ld = 0
    d.data = T_host.data_ptr()
    for A in factors_host:
        if A.is_cuda or A.dtype != torch.float32 or not A.is_contiguous():
            raise NTFError(1, "factors_host must be contiguous host float32 tensors")
    o = (opts or Opts()).c()
    rep = _Report()
    _check(load().ntf_solve_host(C.byref(d), _ptr_array(factors_host), int(factors_host[0].shape[1]), C.byref(o),
                                 C.byref(rep), _stream(stream)))
    return _report(rep)


class Solver:
    """Stateful solver (``ntf_solver_*``): create once, ``run(k)`` asynchronously, ``report()``.
    ``Solver.tucker(X, ...)`` and ``Solver.streamed(T_host, ...)`` build it on Tucker-format data or
    on a tensor that stays in host memory."""

    def __init__(self, T, factors: List, opts: Optional[Opts] = None, dims=None, ld: int = 0, stream=None,
                 _create=None):
        torch = _torch()
        for A in factors:
            _require_cuda(A, "factor", torch.float32)
        self._o = (opts or Opts()).c()
        self._h = C.c_void_p()
        if _create is None:
            self._T = T
            self._d = _tensor_desc(T, dims, ld)
            _check(load().ntf_solver_create(C.byref(self._h), C.byref(self._d), _ptr_array(factors),
                                            int(factors[0].shape[1]), C.byref(self._o), _stream(stream)))
        else:
            self._T = T
            _create(self._h, self._o)
        self.rank = int(factors[0].shape[1])

    @classmethod
    def tucker(cls, X: "Tucker", factors: List, opts: Optional[Opts] = None, stream=None) -> "Solver":
        def create(h, o):
            _check(load().ntf_solver_create_tucker(C.byref(h), C.byref(X.c), _ptr_array(factors),
                                                   int(factors[0].shape[1]), C.byref(o), _stream(stream)))
        return cls(X, factors, opts, stream=stream, _create=create)

    @classmethod
    def streamed(cls, T_host, factors: List, opts: Optional[Opts] = None, slab_rows: int = 0,
                 stream=None) -> "Solver":
        d = _host_desc(T_host)

        def create(h, o):
            _check(load().ntf_solver_create_streamed(C.byref(h), C.byref(d), _ptr_array(factors),
                                                     int(factors[0].shape[1]), C.byref(o), int(slab_rows),
                                                     _stream(stream)))
        return cls((T_host, d), factors, opts, stream=stream, _create=create)

    def run(self, iters: int, stream=None):
        _check(load().ntf_solver_run(self._h, int(iters), _stream(stream)))

    def prepare_graph(self, iters: int, stream=None):
        _check(load().ntf_solver_prepare_graph(self._h, int(iters), _stream(stream)))

    def get_factors(self, factors: List, stream=None):
        _check(load().ntf_solver_get_factors(self._h, _ptr_array(factors), _stream(stream)))

    def report(self, stream=None) -> Report:
        rep = _Report()
        _check(load().ntf_solver_report(self._h, C.byref(rep), _stream(stream)))
        return _report(rep)

    def set_timing(self, every):
        """Time the MTTKRP streams of every ``every``-th iteration (True = 1, False/0 = off)."""
        _check(load().ntf_solver_set_timing(self._h, int(every)))

    def mttkrp_time(self, stream=None):
        ms = C.c_double()
        n = C.c_int64()
        b = C.c_double()
        _check(load().ntf_solver_mttkrp_time(self._h, C.byref(ms), C.byref(n), C.byref(b), _stream(stream)))
        return ms.value, n.value, b.value

    def close(self):
        if self._h:
            load().ntf_solver_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------
# Tucker-format data (Appendix A) and tensors streamed from host memory
# ----------------------------------------------------------------------------
class Tucker:
    """Tucker-format data ``(U_0 (x) ... (x) U_{N-1}) G`` on the device: ``core`` is a float32 CUDA tensor
    of shape (r_0, .., r_{N-1}), ``U`` the float32 CUDA bases (n_p, r_p).  The core is copied into a
    buffer with 16-byte rows (the library's tensor layout)."""

    def __init__(self, core, U: Sequence):
        torch = _torch()
        _require_cuda(core, "core", torch.float32)
        cd = list(core.shape)
        if len(U) != len(cd):
            raise NTFError(1, "one basis per core mode")
        ld = -(-cd[-1] // 4) * 4
        rows = 1
        for v in cd[:-1]:
            rows *= int(v)
        buf = torch.zeros((rows, ld), dtype=torch.float32, device=core.device)
        buf[:, :cd[-1]] = core.reshape(rows, cd[-1])
        self._core = buf
        self.U = []
        for p, u in enumerate(U):
            _require_cuda(u, f"U_{p}", torch.float32)
            if u.dim() != 2 or int(u.shape[1]) != cd[p]:
                raise NTFError(1, f"U_{p} must be (n_{p}, {cd[p]})")
            self.U.append(u)
        self.dims = [int(u.shape[0]) for u in U]
        self.core_dims = cd
        c = _Tucker()
        c.core = _tensor_desc(buf, cd, ld)
        for p, u in enumerate(self.U):
            c.dims[p] = self.dims[p]
            c.U[p] = u.data_ptr()
        self.c = c


def tucker_mttkrp(X: Tucker, factors: Sequence, mode: int, out=None, stream=None):
    """MTTKRP of the Tucker-format tensor through its core (Appendix A)."""
    torch = _torch()
    rank = int(factors[0 if mode != 0 else 1].shape[1])
    dev = X.U[0].device
    if out is None:
        out = torch.empty((X.dims[mode], rank), dtype=torch.float32, device=dev)
    need = int(load().ntf_tucker_mttkrp_workspace_bytes(C.byref(X.c), rank, mode))
    ws = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    ptrs = _ptr_array([None if l == mode else A for l, A in enumerate(factors)])
    _check(load().ntf_tucker_mttkrp(C.byref(X.c), ptrs, rank, mode, _ptr(out), _ptr(ws), ws.numel(), _stream(stream)))
    return out


def tucker_norm_sq(X: Tucker, out=None, stream=None):
    torch = _torch()
    dev = X.U[0].device
    if out is None:
        out = torch.empty((), dtype=torch.float64, device=dev)
    ws = torch.empty(max(int(load().ntf_tucker_norm_workspace_bytes(C.byref(X.c))), 256), dtype=torch.uint8,
                     device=dev)
    _check(load().ntf_tucker_norm_sq(C.byref(X.c), _ptr(out), _ptr(ws), ws.numel(), _stream(stream)))
    return out


def solve_tucker(X: Tucker, factors: List, opts: Optional[Opts] = None, stream=None) -> Report:
    """Alg. 2 (or Alg. 1) on the Tucker-format objective F_t, in place on the CUDA ``factors``."""
    torch = _torch()
    for A in factors:
        _require_cuda(A, "factor", torch.float32)
    o = (opts or Opts()).c()
    rep = _Report()
    _check(load().ntf_solve_tucker(C.byref(X.c), _ptr_array(factors), int(factors[0].shape[1]), C.byref(o),
                                   C.byref(rep), _stream(stream)))
    return _report(rep)


def _host_desc(T_host) -> _Tensor:
    """Describe a contiguous host float32/bfloat16 torch tensor whose last dim gives 16-byte rows."""
    torch = _torch()
    if not isinstance(T_host, torch.Tensor) or T_host.is_cuda or not T_host.is_contiguous():
        raise NTFError(1, "T_host must be a contiguous host tensor")
    d = _Tensor()
    if T_host.dtype == torch.float32:
        d.dtype = NTF_F32
    elif T_host.dtype == torch.bfloat16:
        d.dtype = NTF_BF16
    else:
        raise NTFError(1, "T_host must be float32 or bfloat16")
    d.order = T_host.dim()
    for i, v in enumerate(T_host.shape):
        d.dims[i] = int(v)
    d.ld = 0
    d.data = T_host.data_ptr()
    return d


def mttkrp_streamed(T_host, factors: Sequence, mode: int, out=None, slab_rows: int = 0, stream=None):
    """MTTKRP of a tensor in host memory, streamed to the device by slabs of mode 0."""
    torch = _torch()
    d = _host_desc(T_host)
    rank = int(factors[0 if mode != 0 else 1].shape[1])
    dev = factors[0 if mode != 0 else 1].device
    if out is None:
        out = torch.empty((int(T_host.shape[mode]), rank), dtype=torch.float32, device=dev)
    need = int(load().ntf_mttkrp_streamed_workspace_bytes(C.byref(d), rank, mode, int(slab_rows)))
    ws = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    ptrs = _ptr_array([None if l == mode else A for l, A in enumerate(factors)])
    # the staging buffers in ws are filled on the library's copy stream, but every copy completes
    # before the work on `stream` that reads it, so ws may return to torch's stream-ordered cache
    _check(load().ntf_mttkrp_streamed(C.byref(d), ptrs, rank, mode, _ptr(out), _ptr(ws), ws.numel(), int(slab_rows),
                                      _stream(stream)))
    return out


def solve_streamed(T_host, factors: List, opts: Optional[Opts] = None, slab_rows: int = 0, stream=None) -> Report:
    """Alg. 2 (or Alg. 1) with the tensor in host memory, in place on the CUDA ``factors``."""
    torch = _torch()
    d = _host_desc(T_host)
    for A in factors:
        _require_cuda(A, "factor", torch.float32)
    o = (opts or Opts()).c()
    rep = _Report()
    _check(load().ntf_solve_streamed(C.byref(d), _ptr_array(factors), int(factors[0].shape[1]), C.byref(o),
                                     C.byref(rep), int(slab_rows), _stream(stream)))
    return _report(rep)


from .autograd import CPLoss, cp_loss  # noqa: E402  (re-exported)
