"""Differentiable gain-corrupted correlation (calibration form).

``GainCorr.apply(g, R, V)`` returns L = sum_c ||G R_c G^H - V_c||_F^2 (full
Hermitian matrices held as packed lower triangles); its backward is the
hand-written adjoint kernel in libacf (the forward pass computes the
gradient in the same pass over R and V and keeps it for backward).
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib as A


def _nb_to_n(nb: int) -> int:
    n = int(round(((8 * nb + 1) ** 0.5 - 1) / 2))
    assert n * (n + 1) // 2 == nb
    return n


def gain_loss_and_grad(g: torch.Tensor, R: torch.Tensor, V: torch.Tensor, want_grad: bool = True):
    """g [N] complex64, R/V [C, NB] complex64 on the device -> (loss [], grad [N] complex64)."""
    L = A.lib()
    assert g.is_cuda and R.is_cuda and V.is_cuda
    g = g.contiguous()
    R = R.contiguous()
    V = V.contiguous()
    C, NB = R.shape
    N = _nb_to_n(NB)
    loss = torch.empty((), dtype=torch.float32, device=g.device)
    grad = torch.empty(N, dtype=torch.complex64, device=g.device) if want_grad else None
    st = L.acf_gain_forward(A.ptr(R), A.ptr(V), A.ptr(g), N, C, A.ptr(loss), A.ptr(grad), A.stream_handle())
    A.check(st)
    return loss, grad


def gain_grad(g: torch.Tensor, R: torch.Tensor, V: torch.Tensor):
    L = A.lib()
    C, NB = R.shape
    N = _nb_to_n(NB)
    grad = torch.empty(N, dtype=torch.complex64, device=g.device)
    A.check(L.acf_gain_backward(A.ptr(R.contiguous()), A.ptr(V.contiguous()), A.ptr(g.contiguous()), N, C,
                                A.ptr(grad), A.stream_handle()))
    return grad


class GainCorr(torch.autograd.Function):
    """L(g) = sum_c ||diag(g) R_c diag(g)^H - V_c||_F^2; d/dg by the adjoint kernel.

    The gradient follows torch's convention for a real loss of complex
    inputs: dL/dRe g + i dL/dIm g."""

    @staticmethod
    def forward(ctx, g, R, V):
        loss, grad = gain_loss_and_grad(g.detach(), R.detach(), V.detach(), want_grad=g.requires_grad)
        ctx.save_for_backward(grad if grad is not None else torch.empty(0, device=g.device))
        return loss

    @staticmethod
    def backward(ctx, grad_out):
        (grad,) = ctx.saved_tensors
        return grad_out * grad, None, None
