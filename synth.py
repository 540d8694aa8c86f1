"""Seeded synthetic inputs for nonnegative CP factorization problems.

This module is the only code shared by the FP64 oracle (``oracle/``) and the
CUDA path (``paper_2001_04321_gb300``): it draws ground-truth factors, builds
the noisy data tensor and draws the random initial factors.  It contains none
of the solver's arithmetic (no MTTKRP, Gram, block update, extrapolation or
objective); both sides receive the arrays it returns as plain inputs.

The recipe follows the paper's synthetic-data protocol (Sec. 4.1, "Generate a
synthetic data"): ground-truth factors with i.i.d. U[0,1] entries, the clean
tensor built from them, Gaussian noise added and the result clipped at zero,
``T = max(0, T_clean + sigma * E)``.  Random initial factors are i.i.d. U[0,1]
as in Sec. 4.1 ("Initialization, number of runs and plots").

Readings that are not in the paper:
  * the noise level is *relative*: ``sigma = noise_rel * ||T_clean||_F / sqrt(numel)``;
  * ``recipe="illcond"``: every column of a factor is one shared U[0,1] base
    column plus ``0.05 * U[0,1]`` (an ill-conditioned Gram, cf. Sec. 4.2's
    ill-conditioned experiment, which uses a different mixing rule);
  * ``recipe="sparse30"``: U[0,1] entries with each entry zeroed independently
    with probability 0.3;
  * the tensor is stored C-order, last mode fastest.
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import numpy as np

__all__ = [
    "true_factors",
    "make_tensor",
    "make_init",
    "WORKLOADS",
]


def _rng(seed: int) -> np.random.Generator:
    # PCG64 gives the same stream on x86_64 and aarch64.
    return np.random.Generator(np.random.PCG64(int(seed)))


def true_factors(dims: Sequence[int], rank: int, seed: int,
                 recipe: str = "uniform") -> List[np.ndarray]:
    """Ground-truth factors ``A_true[l]`` of shape ``(dims[l], rank)``, float64."""
    rng = _rng(seed)
    out = []
    for I in dims:
        if recipe == "uniform":
            A = rng.random((I, rank))
        elif recipe == "illcond":
            base = rng.random((I, 1))
            A = base + 0.05 * rng.random((I, rank))
        elif recipe == "sparse30":
            A = rng.random((I, rank))
            A[rng.random((I, rank)) < 0.3] = 0.0
        else:
            raise ValueError(f"unknown recipe {recipe!r}")
        out.append(A)
    return out


def _other_modes_rows(factors: Sequence[np.ndarray]) -> np.ndarray:
    """Rows ``prod_{l>=1} A_l[i_l, p]`` over the C-order multi-index
    ``(i_1, ..., i_{N-1})`` (mode 0 excluded), shape ``(prod I_l, r)``."""
    rows = factors[1]
    for A in factors[2:]:
        rows = (rows[:, None, :] * A[None, :, :]).reshape(-1, A.shape[1])
    return rows


def make_tensor(dims: Sequence[int], rank: int, noise_rel: float, seed: int,
                recipe: str = "uniform", dtype=np.float32,
                chunk_rows: int = 32) -> Tuple[np.ndarray, List[np.ndarray]]:
    """Return ``(T, A_true)``: the noisy nonnegative tensor (``dtype``, C order)
    and its ground-truth factors (float64).

    ``T_clean`` is assembled mode-0 slab by slab (``chunk_rows`` slabs at a
    time) so that a 500^3 tensor needs only one output-sized buffer.
    """
    dims = [int(d) for d in dims]
    if len(dims) < 2:
        raise ValueError("order must be >= 2")
    A = true_factors(dims, rank, seed, recipe)
    rng = _rng(seed + 7919)
    rest = _other_modes_rows(A)                      # (prod_{l>=1} I_l, r)
    I0 = dims[0]
    slab = rest.shape[0]
    T = np.empty((I0, slab), dtype=dtype)
    sq = 0.0
    for s in range(0, I0, chunk_rows):
        e = min(I0, s + chunk_rows)
        block = A[0][s:e] @ rest.T                   # float64 (e-s, slab)
        sq += float(np.einsum("ij,ij->", block, block))
        T[s:e] = block
    sigma = noise_rel * math.sqrt(sq) / math.sqrt(T.size) if noise_rel > 0 else 0.0
    if sigma > 0:
        for s in range(0, I0, chunk_rows):
            e = min(I0, s + chunk_rows)
            noise = rng.standard_normal((e - s, slab))
            T[s:e] = np.maximum(0.0, T[s:e].astype(np.float64) + sigma * noise)
    return T.reshape(dims), A


def make_init(dims: Sequence[int], rank: int, seed: int) -> List[np.ndarray]:
    """Random initial factors, i.i.d. U[0,1], float32, shapes ``(I_l, rank)``."""
    rng = _rng(10_000 + seed)
    return [rng.random((int(I), rank)).astype(np.float32) for I in dims]


# The five synthetic workloads (shape, rank, noise, recipe) used by the tests
# and the benchmark.  Seeds: data 1234 + index, init 42 + run.
WORKLOADS = {
    "cube20_r5": dict(dims=(20, 20, 20), rank=5, noise_rel=1e-2, recipe="uniform", seed=1234),
    "cube100_r10_illcond": dict(dims=(100, 100, 100), rank=10, noise_rel=1e-3, recipe="illcond", seed=1235),
    "cube500_r20": dict(dims=(500, 500, 500), rank=20, noise_rel=1e-2, recipe="uniform", seed=1236),
    "hyper80_r16_sparse30": dict(dims=(80, 80, 80, 80), rank=16, noise_rel=1e-2, recipe="sparse30", seed=1237),
    "cube300_r32": dict(dims=(300, 300, 300), rank=32, noise_rel=1e-2, recipe="uniform", seed=1238),
}


def make_tucker(dims: Sequence[int], cdims: Sequence[int], seed: int, rank: int = 0, noise: float = 0.0,
                dtype=np.float32) -> Tuple[np.ndarray, List[np.ndarray]]:
    """Tucker-format data ``(G, U)`` (Appendix A): a core ``G`` of shape ``cdims``
    and bases ``U_p`` of shape ``(dims[p], cdims[p])`` with i.i.d. U[0,1] entries.
    With ``rank = 0`` the core is i.i.d. U[0,1] too.  With ``rank > 0`` it is the
    superdiagonal core of a rank-``rank`` CP tensor (ones at (q, .., q), q < rank)
    plus ``noise`` times i.i.d. U[0,1], i.e. the Tucker form of a noisy nonnegative
    rank-``rank`` CP tensor whose factors are the first columns of the bases.
    Either way the tensor described is nonnegative.  It stands in for the
    compressed form of a data set too large to hold densely (the paper compresses
    a surveillance video this way; that data set is not available here)."""
    rng = _rng(seed)
    cdims = tuple(int(c) for c in cdims)
    if rank > 0:
        if rank > min(cdims):
            raise ValueError("rank must not exceed the core dims")
        G = noise * rng.random(cdims)
        for q in range(rank):
            G[(q,) * len(cdims)] += 1.0
    else:
        G = rng.random(cdims)
    U = [rng.random((int(d), int(c))).astype(dtype) for d, c in zip(dims, cdims)]
    return G.astype(dtype), U
