"""torch.autograd.Function for the convolution-product expansion.

y = H_m u = C2R( sum_k hhat_k . R2C(w_k . u) ), Eq. 1.4 with the impulse
responses given by their half spectra hhat_k, differentiable with respect to
u, w and hhat.  Forward and backward run in the CUDA library: the backward
calls pce_backward, which gives dL/du by the adjoint apply, and dL/dw,
dL/dhhat from kernels that recompute the per-term spectra R2C(w_k . u)
instead of storing them.  dL/dhhat follows torch's convention for complex
parameters (dL/dRe + i dL/dIm).
"""
from __future__ import annotations

import torch

from .pce import Plan


class ConvolutionProduct(torch.autograd.Function):
    """y = H_m u for u [B, *shape] (or [*shape]), w [m, *shape] float32, hhat complex64
    [m, Ny, Nx/2+1] (2D) or [m, N/2+1] (1D), all on one CUDA device."""

    @staticmethod
    def forward(ctx, u, w, hhat):
        plan = Plan(w.detach().contiguous(), hhat=hhat.detach().contiguous())
        uc = u.detach().contiguous()
        y = plan.apply(uc)
        ctx.plan = plan
        ctx.save_for_backward(uc)
        return y

    @staticmethod
    def backward(ctx, gy):
        (u,) = ctx.saved_tensors
        need_u, need_w, need_h = ctx.needs_input_grad[:3]
        du, dw, dh = ctx.plan.backward(u, gy.contiguous(), need_u, need_w, need_h)
        return du, dw, dh


def convolution_product(u: torch.Tensor, w: torch.Tensor, hhat: torch.Tensor) -> torch.Tensor:
    """Differentiable y = H_m u (see ConvolutionProduct)."""
    return ConvolutionProduct.apply(u, w, hhat)
