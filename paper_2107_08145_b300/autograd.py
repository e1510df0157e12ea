"""torch.autograd binding of the solver: outputs (I_top, J, F, Q_rad) as a
differentiable function of (log chi, S).

The forward pass is rts_solve; the backward pass is rts_adjoint, the
reverse-sweep adjoint of the discrete short-characteristics solve. The
solver is created with log_chi=True, so the library itself forms
chi = exp(log chi); every step of both passes runs in its kernels and torch
only holds the tensors.
"""
from __future__ import annotations

import torch

from . import Solver


class RTSFunction(torch.autograd.Function):
    """RTSFunction.apply(solver, log_chi, S, bottom, top) -> (I_top, J, F, Q).

    solver must have been created with adjoint=True and log_chi=True. log_chi
    and S are CUDA tensors [B, nz, ny, nx] in the solver's dtype."""

    @staticmethod
    def forward(ctx, solver: Solver, log_chi, S, bottom="equal_s", top="zero"):
        if not getattr(solver, "log_chi", False):
            raise ValueError("RTSFunction needs a Solver(..., adjoint=True, log_chi=True)")
        out = solver.solve(log_chi, S, bottom=bottom, top=top)
        ctx.solver = solver
        ctx.bc = (bottom, top)
        ctx.save_for_backward(log_chi, S)
        ctx.set_materialize_grads(False)
        return out["I_top"], out["J"], out["F"], out["Q"]

    @staticmethod
    def backward(ctx, gI_top, gJ, gF, gQ):
        log_chi, S = ctx.saved_tensors
        solver = ctx.solver
        if all(g is None for g in (gI_top, gJ, gF, gQ)):
            return None, None, None, None, None
        g_logchi, g_S = solver.adjoint(log_chi, S, gI_top=gI_top, gJ=gJ, gF=gF, gQ=gQ, bottom=ctx.bc[0],
                                       top=ctx.bc[1])
        return None, g_logchi, g_S, None, None


def rts_apply(solver: Solver, log_chi, S, bottom="equal_s", top="zero"):
    """Differentiable solve: returns (I_top, J, F, Q)."""
    return RTSFunction.apply(solver, log_chi, S, bottom, top)
