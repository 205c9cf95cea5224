"""FP64 reference for the smooth (von Mises-Fisher kernel) mean-shift -- TEST INFRASTRUCTURE.

The kernel family of Eq. 2 with the exponential profile k = exp(kappa * cos)
instead of the flat kernel of Eq. 3/11. Each step moves every seed to the
kernel-weighted mean of all pixels (the dense update of Sec. 3.2.1) and
renormalises it to the unit sphere:

    x_{t+1} = normalise( sum_i exp(kappa * x_t . p_i) p_i ),   t = 0..T-1

Pixels are unconstrained inputs (no renormalisation inside the graph). The
reference gradient is torch float64 autograd through the unrolled loop on the
CPU, a code path independent of the CUDA adjoint.
"""
from __future__ import annotations

import torch


def vmf_forward(P: torch.Tensor, X0: torch.Tensor, kappa: float, T: int) -> torch.Tensor:
    """x_T for every seed. P [N,d], X0 [M,d]; float64 recommended."""
    X = X0
    for _ in range(T):
        W = torch.exp(kappa * (X @ P.T))
        Y = W @ P
        X = Y / torch.linalg.norm(Y, dim=1, keepdim=True)
    return X


def vmf_objective(P: torch.Tensor, X: torch.Tensor, kappa: float) -> torch.Tensor:
    """f(x) = sum_i exp(kappa * x . p_i) per seed (the unnormalised KDE, Eq. 2)."""
    return torch.exp(kappa * (X @ P.T)).sum(dim=1)


def vmf_loss(P, X0, target, kappa: float, T: int) -> torch.Tensor:
    """sum_j || x_T^j - target_j ||^2."""
    return ((vmf_forward(P, X0, kappa, T) - target) ** 2).sum()


def vmf_loss_and_grads(P, X0, target, kappa: float, T: int):
    """(loss, dloss/dP, dloss/dX0) by float64 autograd of the unrolled loop."""
    P = torch.as_tensor(P, dtype=torch.float64).detach().clone().requires_grad_(True)
    X0 = torch.as_tensor(X0, dtype=torch.float64).detach().clone().requires_grad_(True)
    target = torch.as_tensor(target, dtype=torch.float64)
    loss = vmf_loss(P, X0, target, kappa, T)
    gP, gX = torch.autograd.grad(loss, (P, X0))
    return loss.detach(), gP.detach(), gX.detach()


def vmf_vjp(P, X0, kappa: float, T: int, G):
    """(x_T, <G, dx_T/dP>, <G, dx_T/dX0>): the vector-Jacobian product for an
    arbitrary upstream gradient G [M,d], by float64 autograd."""
    P = torch.as_tensor(P, dtype=torch.float64).detach().clone().requires_grad_(True)
    X0 = torch.as_tensor(X0, dtype=torch.float64).detach().clone().requires_grad_(True)
    G = torch.as_tensor(G, dtype=torch.float64)
    XT = vmf_forward(P, X0, kappa, T)
    gP, gX = torch.autograd.grad(XT, (P, X0), grad_outputs=G)
    return XT.detach(), gP.detach(), gX.detach()
