"""torch.autograd.Function over sdf_execute / sdf_backward.

``sdf(points, tau, plan)`` returns the unsigned S grid of ``plan`` for
``points``; its backward calls the hand-written adjoint (sdf_backward), which
gives dL/dY for every point and dL/dtau.  Nodes the forward flagged CAPPED
contribute nothing (their value is a clamp).  The plan must have been created
with the same tau and with grad S among its outputs.
"""
from __future__ import annotations

import torch

from . import Plan


class SDFFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, points, tau, plan: Plan):
        if abs(float(tau) - plan.tau) > 1e-12 * max(1.0, abs(plan.tau)):
            raise ValueError("tau differs from the plan's tau")
        out = plan.execute(points.detach(), None, flags=True)
        ctx.plan = plan
        ctx.save_for_backward(points.detach(), out["S"], out["flags"])
        ctx.tau_dtype = tau.dtype if torch.is_tensor(tau) else torch.float64
        return out["S"]

    @staticmethod
    def backward(ctx, grad_S):
        points, S, flags = ctx.saved_tensors
        dY, dtau = ctx.plan.backward(points, grad_S.to(S.dtype).contiguous(), S, flags)
        return dY.to(points.dtype), dtau.reshape(()).to(ctx.tau_dtype), None


def sdf(points, tau, plan: Plan):
    """Unsigned S on the plan's grid, differentiable in points and tau."""
    return SDFFunction.apply(points, tau, plan)
