"""ln Z/V of a HOTRG run as a differentiable function of beta (torch.autograd).

The forward pass runs the steps in libhotrg.so with the beta-derivative carried in
forward mode (hotrg_set_tangent): after every step the library holds ln Z^(p)/2^p
and its derivative d(ln Z^(p)/2^p)/d beta (Sec. 4.1.1, Eqs. eq_lnZ and
K_recurrence, differentiated through every stage of the step).  The input is the
single scalar beta, so the vector-Jacobian product of the backward pass is the
incoming gradient times that derivative: no tape, no checkpoint of T or of the
isometries.  This module only marshals values between torch and the library.
"""

from __future__ import annotations

import torch

from . import binding as _b


class LnZPerSite(torch.autograd.Function):
    """ln Z^(p)/2^p after each step of a run started from the Ising tensor at (beta, h).

    forward(beta, d, h, chi, axes, precision) -> tensor [len(axes)] (float64, CPU);
    backward gives d/d beta of sum(grad_out * lnz)."""

    @staticmethod
    def forward(ctx, beta, d: int, h: float, chi: int, axes, precision: int = _b.PREC_FP64):
        b = float(beta.detach().cpu().item())
        run = _b.Hotrg(d, b, h, precision=precision)
        lnz, dlnz = [], []
        try:
            _b.hotrg_set_tangent(run.ctx, True)
            for a in axes:
                run.step(int(a), chi)
                lnz.append(run.free_energy()[0])
                dlnz.append(run.energy()[0])
        finally:
            run.close()
        ctx.save_for_backward(torch.tensor(dlnz, dtype=torch.float64))
        return torch.tensor(lnz, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_out):
        (dlnz,) = ctx.saved_tensors
        g = (grad_out.to(torch.float64).cpu() * dlnz).sum()
        return g.reshape(()), None, None, None, None, None


def ln_z_per_site(beta, d: int, h: float, chi: int, axes, precision: int = _b.PREC_FP64):
    """Differentiable ln Z/V per step; `beta` a 0-d float64 tensor (requires_grad for d/d beta)."""
    if not torch.is_tensor(beta):
        beta = torch.tensor(float(beta), dtype=torch.float64)
    return LnZPerSite.apply(beta, d, h, chi, list(axes), precision)


def energy_per_site(beta: float, d: int, h: float, chi: int, axes, precision: int = _b.PREC_FP64):
    """Internal energy per site u = -d(ln Z/V)/d beta after the last step, through autograd."""
    bt = torch.tensor(float(beta), dtype=torch.float64, requires_grad=True)
    lnz = ln_z_per_site(bt, d, h, chi, axes, precision)
    (g,) = torch.autograd.grad(lnz[-1], bt)
    return -float(g)
