"""Differentiable solve x = D[U]^{-1} b (Eq. 1) as a torch.autograd.Function.

Backward, for a real loss L with incoming gradient eta = dL/dRe x + i dL/dIm x
(PyTorch's complex convention):
  grad_b = lam = D^{-dag} eta, one adjoint solve done as gamma5 D^{-1} gamma5 eta
           (gamma5-hermiticity, gamma5 D gamma5 = D^dag);
  grad_U = kappa * bc * M^dag with the colour outer products
           M_mu(x) = sum_spin [ x(x+mu) ((1 - gamma_mu) lam(x))^dag + ((1 + gamma_mu) lam(x+mu)) x(x)^dag ]
           (the fermion-force kernel), from dL = -Re<lam, dD x>.
x is not kept from the forward Krylov iterations: with recompute=True (default)
backward re-solves it in mixed precision from b; otherwise the forward x is saved.
With csw != 0 the link gradient includes the clover term's part (the
derivative of the four-plaquette leaves of F).
"""
from __future__ import annotations

import torch

from . import F32, Gauge, force, solve, solve_opts


class SolveFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, b, gauge, kappa, csw, tol, inner_prec, recompute):
        single = b.dim() == 3
        bb = b.unsqueeze(0) if single else b
        x, _ = solve(gauge, bb.detach(), kappa, csw, tol, solve_opts(inner_prec=inner_prec))
        ctx.gauge, ctx.kappa, ctx.csw, ctx.tol, ctx.inner_prec = gauge, kappa, csw, tol, inner_prec
        ctx.recompute, ctx.single = recompute, single
        if recompute:
            ctx.save_for_backward(bb.detach())
        else:
            ctx.save_for_backward(x)
        return x[0] if single else x

    @staticmethod
    def backward(ctx, grad_x):
        g = ctx.gauge
        eta = grad_x.unsqueeze(0) if ctx.single else grad_x
        eta = eta.contiguous().to(torch.complex128)
        lam, _ = solve(g, eta, ctx.kappa, ctx.csw, ctx.tol, solve_opts(inner_prec=ctx.inner_prec, dagger=True))
        grad_b = lam[0] if ctx.single else lam
        grad_U = None
        if ctx.needs_input_grad[0]:
            (saved,) = ctx.saved_tensors
            if ctx.recompute:
                x, _ = solve(g, saved, ctx.kappa, ctx.csw, ctx.tol, solve_opts(inner_prec=ctx.inner_prec))
            else:
                x = saved
            # summed over the right-hand sides by the force kernel
            grad_U = force(g, x, lam, ctx.kappa, project=False, csw=ctx.csw)
        return grad_U, grad_b, None, None, None, None, None, None


def solve_fn(U: torch.Tensor, b: torch.Tensor, L, kappa: float, csw: float = 0.0, tol: float = 1e-10,
             inner_prec: int = F32, gauge: Gauge = None, bc=(1, 1, 1, -1), recompute: bool = True):
    """x = D[U]^{-1} b with gradients for b and U (Wilson or Wilson-clover).

    U: complex128 [4][V][3][3] CUDA tensor; b: complex128 [V][4][3] or [nrhs][V][4][3].
    gauge: optional prebuilt Gauge for U (with its clover term if csw != 0); it is
    checked against U at a few probe sites and refused (ValueError) if it was
    built from another field."""
    if gauge is None:
        gauge = Gauge(U.detach(), L, bc)
        if csw != 0.0:
            gauge.clover_build(kappa, csw)
    else:
        if U is not None and not gauge.matches(U):
            raise ValueError("gauge was not built from U")
        if csw != 0.0 and gauge.clover != (float(kappa), float(csw)):
            raise ValueError("gauge's clover term was not built with this kappa and csw")
    return SolveFn.apply(U, b, gauge, float(kappa), float(csw), float(tol), int(inner_prec), bool(recompute))
