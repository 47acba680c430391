"""torch.autograd.Function around top_solve / top_grad.

`TopCost.apply(waypoints, durations, solver, workload)` returns the cost of
every trajectory after `workload.max_iters` CADMM iterations (closed-form
step, no inequality rows); its backward runs the library's adjoint through
the unrolled iterations (top_grad) and returns d/d(waypoints) [S+B, 3] and
d/d(durations) [S].  The boundary states, offsets, mode and rho come from the
workload and are held fixed.  Use it for outer time allocation: a loss on the
costs back-propagates into the segment durations.
"""
from __future__ import annotations

import torch

from . import top as _top


class TopCost(torch.autograd.Function):
    @staticmethod
    def forward(ctx, waypoints, durations, solver, workload):
        tensors = solver.device_inputs(workload)
        tensors["waypoints"] = waypoints.detach().to(device="cuda", dtype=torch.float64).contiguous()
        tensors["durations"] = durations.detach().to(device="cuda", dtype=torch.float64).contiguous()
        out = solver.solve(workload, tensors=tensors)
        ctx.solver = solver
        ctx.workload = workload
        ctx.tensors = tensors
        ctx.like = ((waypoints.device, waypoints.dtype), (durations.device, durations.dtype))
        return out["cost"].clone()

    @staticmethod
    def backward(ctx, gcost):
        dw, dT = ctx.solver.grad(ctx.workload, dJ=gcost.detach().to(torch.float64).contiguous(),
                                 tensors=ctx.tensors)
        (dev_w, dt_w), (dev_T, dt_T) = ctx.like  # gradients live where their inputs do
        return dw.to(device=dev_w, dtype=dt_w), dT.to(device=dev_T, dtype=dt_T), None, None


def top_cost(waypoints, durations, solver: "_top.Solver", workload):
    return TopCost.apply(waypoints, durations, solver, workload)
