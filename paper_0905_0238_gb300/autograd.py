"""torch.autograd bindings of the library's adjoints.

``born_misfit(solver, V, layer_vel, D)`` returns J = ||F(c0) V - D||^2 (float64, 0-d) whose
backward gives dJ/dV through the adjoint Born operator and dJ/d(layer velocities) through
the reverse-mode depth march, both computed by the library's CUDA kernels in one call
(``edt_misfit_grad``).

``invert(solver, D, layer_vel=None)`` returns the inverted model V whose backward gives dL/dD
through the adjoint of the damped solve and, when the layer velocities are given, dL/dc
through the solve's dependence on the reference (``edt_invert_vjp``, which reuses the factors
of the forward call; run the backward before the solver inverts again).
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
    """V = S(c) D, the damped inversion of a line-geometry ``Solver`` (EDT_MIXED): linear in D,
    and a function of the layer velocities c through the kernel rows and the damping."""

    @staticmethod
    def forward(ctx, D, layer_vel, solver, out_dtype):
        if layer_vel is not None:
            solver.set_reference(layer_vel.detach().cpu().numpy())
        ctx.solver = solver
        ctx.d_dtype = D.dtype
        ctx.vel_meta = None if layer_vel is None else (layer_vel.device, layer_vel.dtype)
        return solver.invert(D.detach().contiguous(), out_dtype=out_dtype)

    @staticmethod
    def backward(ctx, Vbar):
        want_D = ctx.needs_input_grad[0]
        want_c = ctx.vel_meta is not None and ctx.needs_input_grad[1]
        if not (want_D or want_c):
            return None, None, None, None
        Dbar, gc = ctx.solver.invert_vjp(Vbar.contiguous(), want_D=want_D, want_c=want_c,
                                         out_dtype=ctx.d_dtype)
        if gc is not None:
            gc = gc.to(*ctx.vel_meta)
        return Dbar, gc, None, None


def invert(solver, D, layer_vel=None, out_dtype=None):
    """V = S(c) D, differentiable in D and, given as a tensor, in the layer velocities c (the
    solver's reference is set to them)."""
    return Invert.apply(D, layer_vel, solver, out_dtype or torch.float64)
