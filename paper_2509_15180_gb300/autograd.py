"""``VineSim``: the growth simulation and its adjoint as a torch.autograd.Function.

Forward grows every robot of a batch from one link to its full length with
the given actuator pressures and spans (``vine_set_actuators`` +
``vine_simulate``) and returns a cost per robot: the tip distance
|p_tip - goal| (``vine_grad``), or the path cost (1/N) sum_k |p_k - q_k|^2
of the link end points against target points (``vine_grad_path``).  The
derivatives come from the hand-written adjoint (implicit differentiation at
the final equilibrium) computed in the same forward call, and backward only
applies the chain rule (upstream gradient of each robot's cost times that
robot's derivatives).  All arithmetic of the simulation and the adjoint runs
in ``libvine.so``.
"""
from __future__ import annotations

import torch

from . import vine


class VineSim(torch.autograd.Function):
    """cost = VineSim.apply(act_pressure, act_begin, act_end, batch, goal, kind)

    act_pressure, act_begin, act_end: CUDA float32 tensors [n_act] (Pa, link
    units) in the batch's actuator order; batch: a ``vine.Batch``; goal: CUDA
    float32 [n, 2] goal points (kind "tip") or [total_links, 2] target points
    of the link ends (kind "path").  Returns float64 [n].  Robots whose adjoint is undefined
    (exact Hessian not positive definite at the equilibrium, or no valid
    state) get NaN derivatives; ``VineSim.last_status`` holds the per-robot
    vine_grad status of the last forward."""

    last_status = None

    @staticmethod
    def forward(ctx, act_pressure, act_begin, act_end, batch, goal, kind="tip"):
        stream = torch.cuda.current_stream()
        batch.set_actuators(act_pressure.detach().float(), act_begin.detach().float(), act_end.detach().float(),
                            stream)
        batch.reset(stream)
        batch.simulate(stream)
        if kind not in ("tip", "path"):
            raise ValueError("kind must be 'tip' or 'path'")
        grad = batch.grad if kind == "tip" else batch.grad_path
        out = grad(goal.detach().float(), stream)
        VineSim.last_status = out["status"]
        owner = torch.repeat_interleave(torch.arange(batch.n_inst, device=goal.device),
                                        torch.as_tensor(batch.act_ptr[1:] - batch.act_ptr[:-1], device=goal.device))
        ctx.save_for_backward(out["dP"], out["dB"], out["dE"], owner)
        ctx.dtypes = (act_pressure.dtype, act_begin.dtype, act_end.dtype)
        return out["cost"]

    @staticmethod
    def backward(ctx, g_cost):
        dP, dB, dE, owner = ctx.saved_tensors
        w = g_cost.to(torch.float64)[owner]
        return ((w * dP).to(ctx.dtypes[0]), (w * dB).to(ctx.dtypes[1]), (w * dE).to(ctx.dtypes[2]), None, None,
                None)


def tip_cost(act_pressure, act_begin, act_end, batch: "vine.Batch", goal):
    """Functional form of VineSim.apply for the tip cost."""
    return VineSim.apply(act_pressure, act_begin, act_end, batch, goal, "tip")


def path_cost(act_pressure, act_begin, act_end, batch: "vine.Batch", path):
    """Functional form of VineSim.apply for the path cost."""
    return VineSim.apply(act_pressure, act_begin, act_end, batch, path, "path")
