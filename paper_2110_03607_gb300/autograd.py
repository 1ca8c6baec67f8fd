"""ln Z/V of a HOTRG run as a twice-differentiable function of beta (torch.autograd).

The forward pass runs the steps in libhotrg.so with the beta-derivatives carried in
forward mode (hotrg_set_tangent): after every step the library holds ln Z^(p)/2^p,
its derivative d(ln Z^(p)/2^p)/d beta and, in the FP64 form, its second derivative
(Sec. 4.1.1, Eqs. eq_lnZ and K_recurrence, differentiated through every stage of
the step).  The input is the single scalar beta, so the vector-Jacobian product of
the backward pass is the incoming gradient times that derivative, itself a function
of beta whose own backward multiplies by the second derivative: torch.autograd.grad
with create_graph=True gives d^2(ln Z/V)/d beta^2.  No tape, no checkpoint of T or
of the isometries.  This module only marshals values between torch and the library.
"""

from __future__ import annotations

import torch

from . import binding as _b


class _DLnZ(torch.autograd.Function):
    """d(ln Z/V)/d beta per step as a function of beta, its derivative the second one."""

    @staticmethod
    def forward(ctx, beta, dlnz, d2lnz):
        ctx.save_for_backward(d2lnz)
        ctx.has_d2 = bool(torch.isfinite(d2lnz).all())
        return dlnz.clone()

    @staticmethod
    def backward(ctx, grad_out):
        (d2lnz,) = ctx.saved_tensors
        if not ctx.has_d2:
            raise RuntimeError("the second derivative is carried in the FP64 form only "
                               "(precision PREC_FP64)")
        g = (grad_out.to(torch.float64).cpu() * d2lnz).sum()
        return g.reshape(()), None, None


class LnZPerSite(torch.autograd.Function):
    """ln Z^(p)/2^p after each step of a run started from the Ising tensor at (beta, h).

    forward(beta, d, h, chi, axes, precision, order) -> tensor [len(axes)] (float64, CPU);
    backward gives d/d beta of sum(grad_out * lnz), differentiable once more when
    order = 2 (the second derivative carried; FP64 form)."""

    @staticmethod
    def forward(ctx, beta, d: int, h: float, chi: int, axes, precision: int = _b.PREC_FP64, order: int = 1):
        b = float(beta.detach().cpu().item())
        if order == 2 and precision != _b.PREC_FP64:
            raise ValueError("the second derivative is carried in the FP64 form only")
        second = order == 2
        run = _b.Hotrg(d, b, h, precision=precision)
        lnz, dlnz, d2lnz = [], [], []
        try:
            _b.hotrg_set_tangent(run.ctx, 2 if second else 1)
            for a in axes:
                run.step(int(a), chi)
                lnz.append(run.free_energy()[0])
                dlnz.append(run.energy()[0])
                d2lnz.append(run.specific_heat()[0] if second else float("nan"))
        finally:
            run.close()
        # beta itself (an input): in a double backward it carries the graph to _DLnZ
        ctx.save_for_backward(beta, torch.tensor(dlnz, dtype=torch.float64),
                              torch.tensor(d2lnz, dtype=torch.float64))
        return torch.tensor(lnz, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_out):
        beta, dlnz, d2lnz = ctx.saved_tensors
        d = _DLnZ.apply(beta, dlnz, d2lnz)
        g = (grad_out.to(torch.float64).cpu() * d).sum()
        return g.reshape(()), None, None, None, None, None, None


def ln_z_per_site(beta, d: int, h: float, chi: int, axes, precision: int = _b.PREC_FP64, order: int = 1):
    """Differentiable ln Z/V per step; `beta` a 0-d float64 tensor (requires_grad for d/d beta;
    order = 2 makes the gradient differentiable once more)."""
    if not torch.is_tensor(beta):
        beta = torch.tensor(float(beta), dtype=torch.float64)
    return LnZPerSite.apply(beta, d, h, chi, list(axes), precision, order)


def energy_per_site(beta: float, d: int, h: float, chi: int, axes, precision: int = _b.PREC_FP64):
    """Internal energy per site u = -d(ln Z/V)/d beta after the last step, through autograd."""
    bt = torch.tensor(float(beta), dtype=torch.float64, requires_grad=True)
    lnz = ln_z_per_site(bt, d, h, chi, axes, precision)
    (g,) = torch.autograd.grad(lnz[-1], bt)
    return -float(g)


def specific_heat_per_site(beta: float, d: int, h: float, chi: int, axes):
    """Specific heat per site c = beta^2 d^2(ln Z/V)/d beta^2 after the last step, through
    autograd (double backward; FP64 form)."""
    bt = torch.tensor(float(beta), dtype=torch.float64, requires_grad=True)
    lnz = ln_z_per_site(bt, d, h, chi, axes, _b.PREC_FP64, order=2)
    (g,) = torch.autograd.grad(lnz[-1], bt, create_graph=True)
    (g2,) = torch.autograd.grad(g, bt)
    return float(beta) ** 2 * float(g2)
