"""torch.autograd wrappers of the step and of P -> U, backed by the adjoint
entry points of the CUDA library (kh_step_adjoint, kh_prim_to_cons_adjoint).

Per-step checkpointing: each step saves only its input (U^n, P^n, B^n); the
backward call re-runs that step inside the library and reverses it. The
adiabatic index enters as a 0-d tensor so that its gradient can be
collected; its value must equal the context's.

    from paper_2408_01361_gb300 import autograd as kga
    gam = torch.tensor(cfg["gam"], dtype=torch.float64, device=dev, requires_grad=True)
    U, P, B = kga.prim_to_cons(ctx, P0, B0, gam)
    for _ in range(n):
        U, P, B = kga.step(ctx, U, P, B, gam, dt)
    J = objective(U, P, B); J.backward()

`adj_ctx` (optional): an FP64 context on the same grid whose adjoint is used
when `ctx` runs the mixed-precision step (the gradient is then that of the
FP64 step evaluated along the mixed trajectory).
"""
from __future__ import annotations

import torch


class _PrimToCons(torch.autograd.Function):
    @staticmethod
    def forward(ctx, P, B, gamma, kctx, adj_ctx):
        U = kctx.empty(8)
        kctx.prim_to_cons(P, B, U)
        ctx.save_for_backward(P, B)
        ctx.adj = adj_ctx or kctx
        return U

    @staticmethod
    def backward(ctx, gU):
        P, B = ctx.saved_tensors
        gP, gB, gg = ctx.adj.prim_to_cons_adjoint(P, B, gU.contiguous())
        return gP, gB, torch.tensor(gg, dtype=torch.float64, device=P.device), None, None


class _Step(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, P, B, gamma, kctx, dt, adj_ctx, with_flux):
        U1, P1, B1 = U.clone(), P.clone(), B.clone()
        kctx.step(U1, P1, B1, dt)
        ctx.save_for_backward(U, P, B)
        ctx.adj, ctx.dt, ctx.with_flux = adj_ctx or kctx, float(dt), with_flux
        if with_flux:
            # the stage-2 x1 face fluxes, from the adjoint context's own FP64 step
            a = ctx.adj
            if a is not kctx:
                Ua, Pa, Ba = U.clone(), P.clone(), B.clone()
                a.step(Ua, Pa, Ba, dt)
            F1 = a.stage_flux(1)
            return U1, P1, B1, F1
        return U1, P1, B1

    @staticmethod
    def backward(ctx, gU, gP, gB, gF1=None):
        U, P, B = ctx.saved_tensors

        def c(t):
            return None if t is None else t.contiguous()

        gUi, gPi, gBi, gg = ctx.adj.step_adjoint(U, P, B, ctx.dt, c(gU), c(gP), c(gB), c(gF1))
        return gUi, gPi, gBi, torch.tensor(gg, dtype=torch.float64, device=U.device), None, None, None, None


def prim_to_cons(kctx, P, B, gamma, adj_ctx=None):
    """U = p2c(P, B) with a gradient path to P, B and gamma."""
    _check_gamma(kctx, gamma)
    return _PrimToCons.apply(P, B, gamma, kctx, adj_ctx)


def step(kctx, U, P, B, gamma, dt: float, adj_ctx=None, with_flux: bool = False):
    """One step (kh_step) with a gradient path; with_flux also returns the
    stage-2 x1 face fluxes (8 planes), e.g. for a horizon mass flux."""
    _check_gamma(kctx, gamma)
    return _Step.apply(U, P, B, gamma, kctx, dt, adj_ctx, with_flux)


def _check_gamma(kctx, gamma):
    g = float(gamma.detach().cpu()) if isinstance(gamma, torch.Tensor) else float(gamma)
    if abs(g - float(kctx.cfg["gam"])) > 1e-15 * abs(g):
        raise ValueError("gamma must equal the context's adiabatic index")
