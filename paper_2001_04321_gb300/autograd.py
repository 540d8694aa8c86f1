"""CP loss as a torch.autograd.Function with a hand-written backward.

    loss = (1/2) ||T - [[A_0, ..., A_{N-1}]]||_F^2              (eq. objFun)
         = (1/2) (||T||^2 - 2 <M_{N-1}, A_{N-1}> + sum(V_{N-1} (*) G_{N-1}))
    dloss/dA_n = A_n V_n - M_n                                   (eq. def:grad)

with M_n the MTTKRP of mode n, G_l = A_l^T A_l and V_n the Hadamard product of
the Grams other than n (Appendix A).  The reconstruction is never formed: the
forward is one MTTKRP and N Grams, the backward N-1 more MTTKRPs.  Every step
runs in libntf's kernels; this module only wires them to autograd.  The
tensor T itself receives no gradient; the loss is an FP64 scalar and the
factor gradients are float32 like the factors.
"""
from __future__ import annotations

from typing import List, Optional

import torch

from . import gram, hadamard_grams, mttkrp, objective, tensor_norm_sq, block_gradient, NTFError


class CPLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, T, dims: Optional[List[int]], ld: int, tnorm_sq, *factors):
        if dims is None:
            dims = list(T.shape)
        N = len(dims)
        if len(factors) != N:
            raise NTFError(1, f"CPLoss needs {N} factors, got {len(factors)}")
        F = [A.detach().contiguous() for A in factors]
        grams = [gram(A) for A in F]
        M_last = mttkrp(T, F, N - 1, dims=dims, ld=ld)
        V_last = hadamard_grams(grams, N - 1)
        # ||T||^2 is a property of the data: a caller that evaluates the loss repeatedly on one
        # tensor passes it once (device float64 scalar) and saves a pass over T per forward
        tn = tensor_norm_sq(T, dims=dims, ld=ld) if tnorm_sq is None else tnorm_sq
        f = objective(tn, M_last, F[N - 1], V_last)          # ||T - X||^2 (FP64, device)
        ctx.save_for_backward(T, M_last, *F)
        ctx.grams = grams
        ctx.dims = dims
        ctx.ld = ld
        return 0.5 * f                                        # FP64 scalar

    @staticmethod
    def backward(ctx, grad_out):
        T, M_last, *F = ctx.saved_tensors
        N = len(F)
        g = grad_out.detach().to(torch.float64).reshape(())
        grads = []
        for n in range(N):
            if not ctx.needs_input_grad[4 + n]:
                grads.append(None)
                continue
            M = M_last if n == N - 1 else mttkrp(T, F, n, dims=ctx.dims, ld=ctx.ld)
            V = hadamard_grams(ctx.grams, n)
            grads.append(block_gradient(F[n], M, V, 1.0, scale_dev=g))
        return (None, None, None, None, *grads)


def cp_loss(T, factors, dims=None, ld: int = 0, tnorm_sq=None):
    """(1/2)||T - [[factors]]||^2 with a hand-written MTTKRP backward.  ``tnorm_sq``: optional
    precomputed ||T||^2 (device float64 scalar, e.g. from ``tensor_norm_sq``)."""
    return CPLoss.apply(T, dims, ld, tnorm_sq, *factors)
