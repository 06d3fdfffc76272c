"""torch.autograd.Function for the marginal log-likelihood over the rotation window.

    l(x, kappa, eta) = sum_j log sum_l rho_l (pi sigma^2)^{-M} exp(-||x o e^{-i k theta_l} - y_j||^2 / sigma^2)
    log rho_l        = kappa cos theta_l + eta_l - log sum_window exp(kappa cos theta + eta)

Forward and backward both call mra_loglik_grad: the backward pass recomputes
the posterior in one more sweep over y instead of storing the N x Lw weights.
The gradient with respect to x is returned in torch's convention for a real
loss of a complex input, dl/dRe x + i dl/dIm x.
"""
from __future__ import annotations

import torch

from . import mra


class MarginalLogLik(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, eta, kappa, y, shift, d, Lw, l0, ws, step):
        ll = torch.empty(1, dtype=torch.float64, device=y.device)
        mra.mra_loglik_grad(d, Lw, l0, y, shift, x.detach().contiguous(), eta.detach().contiguous(),
                            float(kappa.detach().item()), ll, None, None, None, ws, step=step)
        ctx.save_for_backward(x, eta, kappa)
        ctx.extra = (y, shift, d, Lw, l0, ws, step)
        return ll[0]

    @staticmethod
    def backward(ctx, g):
        x, eta, kappa = ctx.saved_tensors
        y, shift, d, Lw, l0, ws, step = ctx.extra
        ll = torch.empty(1, dtype=torch.float64, device=y.device)
        dx = torch.empty_like(x)
        de = torch.empty_like(eta)
        dk = torch.empty(1, dtype=torch.float64, device=y.device)
        mra.mra_loglik_grad(d, Lw, l0, y, shift, x.detach().contiguous(), eta.detach().contiguous(),
                            float(kappa.detach().item()), ll, dx, de, dk, ws, step=step)
        return g * dx, g * de, (g * dk).reshape(kappa.shape), None, None, None, None, None, None, None


def marginal_loglik(x, eta, kappa, y, d, Lw, l0=None, shift=None, ws=None, step=1.0):
    """step: spacing of the window's rotations in grid units (theta_l = 2 pi step (l0 + l) / L)."""
    if l0 is None:
        l0 = -(Lw // 2)
    if ws is None:
        ws = mra.workspace(mra.mra_em_workspace_bytes(d, Lw), y.device)
    return MarginalLogLik.apply(x, eta, kappa, y, shift, d, Lw, l0, ws, float(step))
