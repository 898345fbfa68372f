"""The CP reconstruction loss as a ``torch.autograd.Function``.

    loss(A^(1), ..., A^(N)) = ||X - [[A^(1), ..., A^(N)]]||_F^2

(the objective of Eq. (2.3) without its factor 1/2).  The forward pass is the
direct FP64 reconstruction of ``cp_residual_sums``; the hand-written backward
is Algorithm 1's gradient line, dloss/dA^(n) = 2 (A^(n) Gamma^(n,n) - M^(n)),
whose N MTTKRPs come from one fused all-mode dimension-tree pass over X
(``cp_gradient``), on the tensor cores (``prec="bf16x3"``) or in FP64.

Both passes run in the CUDA library; the Function only marshals tensors and
applies the chain-rule scale of the incoming gradient.
"""
from __future__ import annotations

import torch

from . import api

_handles: dict = {}


def _handle_for(device: torch.device) -> api.Handle:
    idx = device.index if device.index is not None else torch.cuda.current_device()
    h = _handles.get(idx)
    if h is None:
        h = api.Handle(idx)
        _handles[idx] = h
    return h


class CPLoss(torch.autograd.Function):
    """loss = ||X - [[A]]||_F^2; backward by the fused MTTKRP.

    X: CUDA tensor (float32 or float64, C-contiguous, order N); factors:
    float64 CUDA tensors of shape (s_n, R).  X receives no gradient.
    """

    @staticmethod
    def forward(ctx, X, handle, prec, *factors):
        A = [f.detach().contiguous() for f in factors]
        # X may be a new tensor at a reused address: the backward's bf16 split of X is rebuilt
        handle.bump_version(X)
        sq_err, _ = api.cp_residual_sums(handle, X, A)
        ctx.save_for_backward(X, *A)
        ctx.handle, ctx.prec = handle, prec
        return torch.tensor(sq_err, dtype=torch.float64, device=X.device)

    @staticmethod
    def backward(ctx, grad_out):
        X, *A = ctx.saved_tensors
        G, _, _ = api.cp_gradient(ctx.handle, X, A, prec=ctx.prec)
        scale = 2.0 * grad_out
        grads = [g.mul_(scale) if ctx.needs_input_grad[3 + n] else None for n, g in enumerate(G)]
        return (None, None, None, *grads)


def cp_loss(X: torch.Tensor, factors, prec: str = "bf16x3", handle: api.Handle | None = None) -> torch.Tensor:
    """||X - [[factors]]||_F^2 as a 0-dim float64 tensor with a fused-MTTKRP backward."""
    if not X.is_cuda:
        raise ValueError("cp_loss: X must be a CUDA tensor")
    for n, f in enumerate(factors):
        if f.dtype != torch.float64 or not f.is_cuda or f.dim() != 2 or f.shape[0] != X.shape[n]:
            raise ValueError(f"cp_loss: factor {n} must be a float64 CUDA tensor of shape ({X.shape[n]}, R)")
    h = handle if handle is not None else _handle_for(X.device)
    return CPLoss.apply(X, h, prec, *factors)
