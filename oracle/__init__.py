"""FP64 CPU oracle for HER-accelerated BCD on dense nonnegative CP factorization.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline / ``--impl reference`` legs of ``bench.py``.  The
product package never imports it.  The arithmetic lives in ``ntf_oracle.c``
(plain C, FP64); this module compiles it with gcc on first use and wraps it
with ctypes so that callers pass numpy arrays.

Every function states the passage of arXiv 2001.04321 it follows.  Modes are
0-based (the paper's mode i is mode i-1 here); tensors are C-order with the
last mode fastest; factors are ``(I_l, r)`` row-major; objectives are
``||T - X||_F^2`` (twice the paper's F of eq. objFun).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ntf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = C.POINTER(C.c_double)
_I64 = C.POINTER(C.c_int64)


def build(force: bool = False) -> str:
    """Compile ``ntf_oracle.c`` into ``liboracle.so`` (gcc, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            lib.oracle_mttkrp.argtypes = [C.c_int, _I64, _D, C.POINTER(_D), C.c_int, C.c_int, _D]
            lib.oracle_mttkrp_kr.argtypes = lib.oracle_mttkrp.argtypes
            lib.oracle_cp_gradient.argtypes = lib.oracle_mttkrp.argtypes
            lib.oracle_gram.argtypes = [_D, C.c_int64, C.c_int, _D]
            lib.oracle_hadamard_grams.argtypes = [C.POINTER(_D), C.c_int, C.c_int, C.c_int, _D]
            lib.oracle_norm_sq.argtypes = [_D, C.c_int64]
            lib.oracle_norm_sq.restype = C.c_double
            lib.oracle_objective_explicit.argtypes = [C.c_int, _I64, _D, C.POINTER(_D), C.c_int]
            lib.oracle_objective_explicit.restype = C.c_double
            lib.oracle_objective_identity.argtypes = [C.c_double, _D, _D, C.c_int64, C.c_int, _D]
            lib.oracle_objective_identity.restype = C.c_double
            lib.oracle_hals.argtypes = [_D, C.c_int64, C.c_int, _D, _D, C.c_int, C.c_double]
            lib.oracle_pgd.argtypes = lib.oracle_hals.argtypes
            lib.oracle_nesterov.argtypes = lib.oracle_hals.argtypes
            lib.oracle_lambda_max.argtypes = [_D, C.c_int]
            lib.oracle_lambda_max.restype = C.c_double
            lib.oracle_extrapolate.argtypes = [_D, _D, C.c_double, C.c_int64, _D]
            lib.oracle_extrapolate.restype = None
            lib.oracle_her_decide.argtypes = [_D, C.c_double, C.c_double, C.c_double, C.c_double]
            tail = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_int,
                    C.c_double, C.c_double, C.c_double, C.c_double,
                    _D, _D, _D, C.POINTER(C.c_int), _D, _D, _D, _D, C.POINTER(C.c_int)]
            lib.oracle_solve.argtypes = [C.c_int, _I64, _D, C.POINTER(_D), C.c_int] + tail
            lib.oracle_solve_tucker.argtypes = [C.c_int, _I64, _I64, _D, C.POINTER(_D), C.POINTER(_D),
                                                C.c_int] + tail
            lib.oracle_tucker_expand.argtypes = [C.c_int, _I64, _I64, _D, C.POINTER(_D), _D]
            lib.oracle_tucker_mttkrp.argtypes = [C.c_int, _I64, _I64, _D, C.POINTER(_D), C.POINTER(_D),
                                                 C.c_int, C.c_int, _D]
            lib.oracle_tucker_norm_sq.argtypes = [C.c_int, _I64, _I64, _D, C.POINTER(_D)]
            lib.oracle_tucker_norm_sq.restype = C.c_double
            lib.oracle_round_bf16.argtypes = [C.POINTER(C.c_float), C.POINTER(C.c_uint16), C.c_int64]
            lib.oracle_round_bf16.restype = None
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _dims(T: np.ndarray):
    d = np.asarray(T.shape, dtype=np.int64)
    return d, d.ctypes.data_as(_I64)


def _ptr_array(arrs: Sequence[np.ndarray]):
    arr = (_D * len(arrs))()
    for i, a in enumerate(arrs):
        arr[i] = _ptr(a)
    return arr


def mttkrp(T, factors, mode: int) -> np.ndarray:
    """MTTKRP of ``mode`` by its entrywise definition (Sec. 2, eq. def:grad)."""
    lib = _load()
    T = _f64(T)
    F = [_f64(A) for A in factors]
    r = F[0].shape[1]
    d, dp = _dims(T)
    M = np.zeros((T.shape[mode], r))
    rc = lib.oracle_mttkrp(T.ndim, dp, _ptr(T), _ptr_array(F), r, mode, _ptr(M))
    if rc:
        raise ValueError("oracle_mttkrp: bad arguments")
    return M


def mttkrp_kr(T, factors, mode: int) -> np.ndarray:
    """MTTKRP via the explicit Khatri-Rao matrix B^n and unfolding T_[n]
    (Sec. 2, eqs. unfold/lrunfold, def:B).  Tiny inputs only."""
    lib = _load()
    T = _f64(T)
    F = [_f64(A) for A in factors]
    r = F[0].shape[1]
    d, dp = _dims(T)
    M = np.zeros((T.shape[mode], r))
    rc = lib.oracle_mttkrp_kr(T.ndim, dp, _ptr(T), _ptr_array(F), r, mode, _ptr(M))
    if rc:
        raise ValueError("oracle_mttkrp_kr: bad arguments")
    return M


def gram(A) -> np.ndarray:
    """``A^T A``."""
    lib = _load()
    A = _f64(A)
    r = A.shape[1]
    G = np.zeros((r, r))
    lib.oracle_gram(_ptr(A), A.shape[0], r, _ptr(G))
    return G


def hadamard_grams(grams: Sequence[np.ndarray], skip: int) -> np.ndarray:
    """Hadamard product of the Grams over ``l != skip`` (Appendix A)."""
    lib = _load()
    G = [_f64(g) for g in grams]
    r = G[0].shape[0]
    V = np.zeros((r, r))
    lib.oracle_hadamard_grams(_ptr_array(G), len(G), skip, r, _ptr(V))
    return V


def norm_sq(T) -> float:
    T = _f64(T)
    return float(_load().oracle_norm_sq(_ptr(T), T.size))


def objective_explicit(T, factors) -> float:
    """``||T - [[A]]||_F^2`` with the reconstruction formed entrywise."""
    lib = _load()
    T = _f64(T)
    F = [_f64(A) for A in factors]
    d, dp = _dims(T)
    return float(lib.oracle_objective_explicit(T.ndim, dp, _ptr(T), _ptr_array(F), F[0].shape[1]))


def cp_gradient(T, factors, mode: int) -> np.ndarray:
    """Gradient of ``(1/2)||T - [[A]]||_F^2`` with respect to factor ``mode``:
    the MTTKRP of the explicitly formed residual ``X - T`` (Sec. 2, eq. def:grad)."""
    lib = _load()
    T = _f64(T)
    F = [_f64(A) for A in factors]
    r = F[0].shape[1]
    d, dp = _dims(T)
    g = np.zeros((T.shape[mode], r))
    rc = lib.oracle_cp_gradient(T.ndim, dp, _ptr(T), _ptr_array(F), r, mode, _ptr(g))
    if rc:
        raise ValueError("oracle_cp_gradient: bad arguments")
    return g


def objective_identity(tnorm_sq: float, M, A, V) -> float:
    """``||T||^2 - 2<M, A> + sum(V (*) A^T A)`` (Sec. 3.1, restart mechanism)."""
    M = _f64(M)
    A = _f64(A)
    V = _f64(V)
    return float(_load().oracle_objective_identity(tnorm_sq, _ptr(M), _ptr(A), A.shape[0],
                                                   A.shape[1], _ptr(V)))


def hals(A, M, V, inner_max: int = 1, inner_tol: float = 1e-2):
    """HALS column sweeps (Sec. 2.1.4) on a copy of ``A``; returns (A_new, sweeps)."""
    A = _f64(A).copy()
    M = _f64(M)
    V = _f64(V)
    s = _load().oracle_hals(_ptr(A), A.shape[0], A.shape[1], _ptr(M), _ptr(V), inner_max, inner_tol)
    return A, s


def pgd(A, M, V, inner_max: int = 1, inner_tol: float = 1e-2):
    """Projected gradient steps with step 1/lambda_max(V) (Sec. 2.2); returns (A_new, steps)."""
    A = _f64(A).copy()
    M = _f64(M)
    V = _f64(V)
    s = _load().oracle_pgd(_ptr(A), A.shape[0], A.shape[1], _ptr(M), _ptr(V), inner_max, inner_tol)
    return A, s


def nesterov(A, M, V, inner_max: int = 1, inner_tol: float = 1e-2):
    """AO-Nesterov block update (Sec. 2.1; momentum sequence t_k of Appendix B,
    projected gradient step of eq. projgrad) on a copy of ``A``; returns (A_new, steps)."""
    A = _f64(A).copy()
    M = _f64(M)
    V = _f64(V)
    s = _load().oracle_nesterov(_ptr(A), A.shape[0], A.shape[1], _ptr(M), _ptr(V), inner_max, inner_tol)
    return A, s


def lambda_max(V) -> float:
    """Largest eigenvalue of a symmetric matrix by cyclic Jacobi rotations."""
    V = _f64(V)
    return float(_load().oracle_lambda_max(_ptr(V), V.shape[0]))


def extrapolate(A, A_prev, beta: float) -> np.ndarray:
    """``max(0, A + beta (A - A_prev))`` (Alg. 2, eq. extproj_her)."""
    A = _f64(A)
    P = _f64(A_prev)
    out = np.empty_like(A)
    _load().oracle_extrapolate(_ptr(A), _ptr(P), float(beta), A.size, _ptr(out))
    return out


def her_decide(state: List[float], f_hat: float, gamma=1.05, gamma_bar=1.01, eta=1.5) -> int:
    """One restart/accept decision of Alg. 2; ``state = [beta, beta_bar, f_hat_prev]``
    is updated in place.  Returns 1 on restart."""
    s = np.asarray(state, dtype=np.float64)
    rc = _load().oracle_her_decide(_ptr(s), float(f_hat), gamma, gamma_bar, eta)
    state[:] = list(s)
    return int(rc)


def round_bf16(x) -> np.ndarray:
    """FP32 -> bfloat16 bits, round to nearest even (uint16 array)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty(x.shape, dtype=np.uint16)
    _load().oracle_round_bf16(x.ctypes.data_as(C.POINTER(C.c_float)),
                              out.ctypes.data_as(C.POINTER(C.c_uint16)), x.size)
    return out


def bf16_to_f64(bits) -> np.ndarray:
    """Exact value of bfloat16 bit patterns."""
    b = np.ascontiguousarray(bits, dtype=np.uint16).astype(np.uint32) << 16
    return b.view(np.float32).astype(np.float64)


class SolveTrace:
    def __init__(self, iters: int, dims, r: int, track_factors: bool):
        order = len(dims)
        self.dims = [int(d) for d in dims]
        self.r = r
        self.fhat = np.zeros(iters)
        self.beta = np.zeros(iters)
        self.beta_bar = np.zeros(iters)
        self.restart = np.zeros(iters, dtype=np.int32)
        self.ftrue = np.zeros(iters)
        self.fblock = np.zeros(iters * order)
        self.fhat0 = np.zeros(1)
        S = sum(self.dims) * r
        self._fac = np.zeros(iters * 3 * S) if track_factors else None

    def _factors(self, k: int, which: int):
        S = sum(self.dims) * self.r
        flat = self._fac[(k - 1) * 3 * S + which * S:(k - 1) * 3 * S + (which + 1) * S]
        out, o = [], 0
        for d in self.dims:
            out.append(flat[o:o + d * self.r].reshape(d, self.r))
            o += d * self.r
        return out

    def A_updated(self, k: int):
        """Factors A^l_k right after the block updates of iteration k (1-based)."""
        return self._factors(k, 0)

    def A_hat(self, k: int):
        """Extrapolated factors A_hat^l_k of iteration k before the restart decision."""
        return self._factors(k, 1)

    def A_after(self, k: int):
        """Factors A^l_k after iteration k's restart decision."""
        return self._factors(k, 2)


_METHODS = {"hals": 0, "pgd": 1, "nesterov": 2}


def _solve_common(fn, prefix, dims, init, iters, her, method, inner_max, inner_tol, beta0, gamma,
                  gamma_bar, eta, track_true, track_blocks, track_factors, force=None):
    F = [_f64(A).copy() for A in init]
    if force is not None:
        force = np.ascontiguousarray(force, dtype=np.int32)
        if force.shape != (iters,):
            raise ValueError("force needs one entry per iteration")
    r = F[0].shape[1]
    tr = SolveTrace(iters, dims, r, track_factors)
    rc = fn(*prefix, _ptr_array(F), r, int(her), _METHODS[method], inner_max, inner_tol, iters,
            beta0, gamma, gamma_bar, eta,
            _ptr(tr.fhat), _ptr(tr.beta), _ptr(tr.beta_bar),
            tr.restart.ctypes.data_as(C.POINTER(C.c_int)),
            _ptr(tr.ftrue) if track_true else None,
            _ptr(tr.fblock) if track_blocks else None,
            _ptr(tr.fhat0),
            _ptr(tr._fac) if track_factors else None,
            force.ctypes.data_as(C.POINTER(C.c_int)) if force is not None else None)
    if rc:
        raise ValueError("oracle solve: bad arguments")
    return F, tr


def solve(T, init, iters: int, her: bool = True, method: str = "hals", inner_max: int = 1,
          inner_tol: float = 1e-2, beta0: float = 0.5, gamma: float = 1.05,
          gamma_bar: float = 1.01, eta: float = 1.5, track_true: bool = False,
          track_blocks: bool = False, track_factors: bool = False, force=None):
    """Alg. 1 (``her=False``) or Alg. 2 (``her=True``) in FP64 from ``init``.
    ``method`` is "hals", "pgd" or "nesterov".  ``force``: optional per-iteration -1 / 0 / 1
    (take Alg. 2's accept or restart branch at that iteration whatever F-hat says).

    Returns ``(factors, trace)``; ``trace.fhat[k-1]`` is F-hat_k (the value Alg. 2's restart test compares),
    ``trace.ftrue[k-1]`` the explicit objective at A_k when ``track_true``; with ``track_factors``
    the trace also holds every iteration's factors (``A_updated``, ``A_hat``, ``A_after``).
    """
    lib = _load()
    T = _f64(T)
    d, dp = _dims(T)
    return _solve_common(lib.oracle_solve, (T.ndim, dp, _ptr(T)), T.shape, init, iters, her, method,
                         inner_max, inner_tol, beta0, gamma, gamma_bar, eta, track_true, track_blocks,
                         track_factors, force)


# --- Tucker-format data (Appendix A) -----------------------------------------

def _tucker_args(G, U):
    G = _f64(G)
    U = [_f64(u) for u in U]
    dims = np.asarray([u.shape[0] for u in U], dtype=np.int64)
    cdims = np.asarray(G.shape, dtype=np.int64)
    if len(U) != G.ndim or any(u.shape[1] != c for u, c in zip(U, G.shape)):
        raise ValueError("U_p must be dims[p] x G.shape[p]")
    return G, U, dims, cdims


def tucker_expand(G, U) -> np.ndarray:
    """The tensor ``(U_0 (x) ... (x) U_{N-1}) G`` written out entry by entry (tiny inputs)."""
    G, U, dims, cdims = _tucker_args(G, U)
    T = np.zeros(tuple(int(x) for x in dims))
    rc = _load().oracle_tucker_expand(G.ndim, dims.ctypes.data_as(_I64), cdims.ctypes.data_as(_I64), _ptr(G),
                                      _ptr_array(U), _ptr(T))
    if rc:
        raise ValueError("oracle_tucker_expand: bad arguments")
    return T


def tucker_mttkrp(G, U, factors, mode: int) -> np.ndarray:
    """MTTKRP of the Tucker-format tensor through its core (Appendix A):
    ``U_n MTTKRP(G, {U_p^T A_p}, n)``."""
    G, U, dims, cdims = _tucker_args(G, U)
    F = [_f64(A) for A in factors]          # factors[mode] is not read
    r = F[0 if mode != 0 else 1].shape[1]
    M = np.zeros((int(dims[mode]), r))
    rc = _load().oracle_tucker_mttkrp(G.ndim, dims.ctypes.data_as(_I64), cdims.ctypes.data_as(_I64), _ptr(G),
                                      _ptr_array(U), _ptr_array(F), r, mode, _ptr(M))
    if rc:
        raise ValueError("oracle_tucker_mttkrp: bad arguments")
    return M


def tucker_norm_sq(G, U) -> float:
    """``||(U_0 (x) ... (x) U_{N-1}) G||_F^2`` through the core and the Grams of U_p."""
    G, U, dims, cdims = _tucker_args(G, U)
    return float(_load().oracle_tucker_norm_sq(G.ndim, dims.ctypes.data_as(_I64), cdims.ctypes.data_as(_I64),
                                               _ptr(G), _ptr_array(U)))


def solve_tucker(G, U, init, iters: int, her: bool = True, method: str = "hals", inner_max: int = 1,
                 inner_tol: float = 1e-2, beta0: float = 0.5, gamma: float = 1.05,
                 gamma_bar: float = 1.01, eta: float = 1.5, track_true: bool = False,
                 track_blocks: bool = False, track_factors: bool = False, force=None):
    """Alg. 1 / Alg. 2 on the Tucker-format objective F_t of Appendix A (eq. objFunTucker)."""
    lib = _load()
    G, U, dims, cdims = _tucker_args(G, U)
    return _solve_common(lib.oracle_solve_tucker,
                         (G.ndim, dims.ctypes.data_as(_I64), cdims.ctypes.data_as(_I64), _ptr(G), _ptr_array(U)),
                         [int(x) for x in dims], init, iters, her, method, inner_max, inner_tol, beta0, gamma,
                         gamma_bar, eta, track_true, track_blocks, track_factors, force)
