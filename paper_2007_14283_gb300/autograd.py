"""torch.autograd.Function over the library's smooth-kernel mean-shift.

VMFMeanShift.apply(P, X0, kappa, T) returns x_T of T unrolled steps
x <- normalise(sum_i exp(kappa (x . p_i - 1)) p_i) computed by
ms_vmf_forward; its backward calls the hand-written adjoint ms_vmf_backward,
which recomputes the iterates instead of saving them. Only P and X0 are saved
for backward.
"""
from __future__ import annotations

import torch

from . import MS_FP32, ms_vmf_backward, ms_vmf_forward


class VMFMeanShift(torch.autograd.Function):
    @staticmethod
    def forward(ctx, P: torch.Tensor, X0: torch.Tensor, kappa: float, T: int, precision: int = MS_FP32) -> torch.Tensor:
        P = P.contiguous()
        X0 = X0.contiguous()
        ctx.save_for_backward(P, X0)
        ctx.kappa = float(kappa)
        ctx.T = int(T)
        ctx.precision = int(precision)
        return ms_vmf_forward(P, X0, kappa, T, precision=precision)

    @staticmethod
    def backward(ctx, GT: torch.Tensor):
        P, X0 = ctx.saved_tensors
        dP, dX0 = ms_vmf_backward(P, X0, ctx.kappa, ctx.T, GT.contiguous(), precision=ctx.precision)
        return (dP if ctx.needs_input_grad[0] else None, dX0 if ctx.needs_input_grad[1] else None, None, None, None)


def vmf_mean_shift(P: torch.Tensor, X0: torch.Tensor, kappa: float = 20.0, T: int = 10,
                   precision: int = MS_FP32) -> torch.Tensor:
    """precision MS_BF16 runs the forward steps (and the backward's recomputed
    iterates) on the tensor cores; the adjoint passes are FP32."""
    return VMFMeanShift.apply(P, X0, kappa, T, precision)
