"""torch.autograd bindings of the library's adjoints.

``born_misfit(solver, V, layer_vel, D)`` returns J = ||F(c0) V - D||^2 (float64, 0-d) whose
backward gives dJ/dV through the adjoint Born operator and dJ/d(layer velocities) through
the reverse-mode depth march, both computed by the library's CUDA kernels in one call
(``edt_misfit_grad``).

``invert(solver, D)`` returns the inverted model V whose backward gives dL/dD through the
adjoint of the damped solve (``edt_invert_adjoint``, which reuses the factors of the forward
call; run the backward before the solver inverts with another reference).
"""
from __future__ import annotations

import torch


class BornMisfit(torch.autograd.Function):
    """J(V, c) = ||F(c) V - D||^2 for a line-geometry ``Solver`` (EDT_MIXED)."""

    @staticmethod
    def forward(ctx, V, layer_vel, D, solver):
        solver.set_reference(layer_vel.detach().cpu().numpy())
        J, gV, gc = solver.misfit_grad(V.detach().contiguous(), D.detach().contiguous())
        ctx.save_for_backward(gV, gc.to(layer_vel.device, layer_vel.dtype))
        return J

    @staticmethod
    def backward(ctx, gJ):
        gV, gc = ctx.saved_tensors
        gV_out = (gJ.to(gV.dtype) * gV) if ctx.needs_input_grad[0] else None
        gc_out = (gJ.to(gc.device, gc.dtype) * gc) if ctx.needs_input_grad[1] else None
        return gV_out, gc_out, None, None


def born_misfit(solver, V, layer_vel, D):
    """J = ||F(layer_vel) V - D||^2, differentiable in V and in the layer velocities."""
    return BornMisfit.apply(V, layer_vel, D, solver)


class Invert(torch.autograd.Function):
    """V = S D, the damped inversion of a line-geometry ``Solver`` (EDT_MIXED)."""

    @staticmethod
    def forward(ctx, D, solver, out_dtype):
        ctx.solver = solver
        ctx.d_dtype = D.dtype
        return solver.invert(D.detach().contiguous(), out_dtype=out_dtype)

    @staticmethod
    def backward(ctx, Vbar):
        Dbar = ctx.solver.invert_adjoint(Vbar.contiguous(), out_dtype=ctx.d_dtype)
        return Dbar, None, None


def invert(solver, D, out_dtype=None):
    """V = S D, differentiable in D (the inversion is linear in the data)."""
    return Invert.apply(D, solver, out_dtype or torch.float64)
