"""torch.autograd wrappers of the rollout and of one step.

The forward and backward passes run in the CUDA library (sim_rollout /
sim_backward, sim_step / sim_step_backward); torch only routes cotangents.
"""
from __future__ import annotations

import torch

from .binding import Simulator


class DiffSimRollout(torch.autograd.Function):
    """(r_ctrl [T,NM], depth [T,NM,Rc], lidar [T,NM,Rl], s_T [NM,D]) =
    rollout(actions [T,NM,A], s_0 [NM,D]) over the simulator's horizon.
    Backpropagation through time is the library's hand-written adjoint with
    segment checkpointing.  The handle keeps the rollout's records, so
    backward must run before the next rollout on the same simulator."""

    @staticmethod
    def forward(ctx, sim: Simulator, actions, s0):
        actions = actions.detach().contiguous()
        sim.reset(s0.detach().contiguous())
        o = sim.rollout(actions)
        sT = sim.get_state()
        ctx.sim = sim
        ctx.actions = actions  # the adjoint re-reads the actions buffer
        empty = actions.new_zeros((sim.T, sim.NM, 0))
        depth = o["depth"] if o["depth"] is not None else empty
        lidar = o["lidar"] if o["lidar"] is not None else empty
        ctx.has = (o["depth"] is not None, o["lidar"] is not None)
        return o["r_ctrl"], depth, lidar, sT

    @staticmethod
    def backward(ctx, g_r, g_depth, g_lidar, g_sT):
        sim = ctx.sim
        if g_r is None:
            g_r = torch.zeros(sim.T, sim.NM, device=sim.device)
        g_depth = g_depth if ctx.has[0] else None
        g_lidar = g_lidar if ctx.has[1] else None
        g_a, g_s0 = sim.backward(g_r, g_depth, g_lidar, g_sT)
        return None, g_a, g_s0


class DiffSimStep(torch.autograd.Function):
    """(s_next [NM,D], r_ctrl [NM], depth [NM,Rc], lidar [NM,Rl]) =
    step(s_t [NM,D], a_t [NM,A]): one differentiable step for closed-loop
    training, where each action depends on the previous observation."""

    @staticmethod
    def forward(ctx, sim: Simulator, s_t, a_t):
        s_t = s_t.detach().contiguous()
        a_t = a_t.detach().contiguous()
        sim.set_state(s_t)
        o = sim.step(a_t)
        s_next = sim.get_state()
        ctx.sim = sim
        ctx.save_for_backward(s_t, a_t, o["done"])
        ctx.has = (o["depth"] is not None, o["lidar"] is not None)
        empty = s_t.new_zeros((sim.NM, 0))
        depth = o["depth"] if o["depth"] is not None else empty
        lidar = o["lidar"] if o["lidar"] is not None else empty
        ctx.mark_non_differentiable(o["done"])
        return s_next, o["r_ctrl"], depth, lidar, o["done"]

    @staticmethod
    def backward(ctx, g_s_next, g_r, g_depth, g_lidar, _g_done):
        sim = ctx.sim
        s_t, a_t, done = ctx.saved_tensors
        if g_r is None:
            g_r = torch.zeros(sim.NM, device=sim.device)
        g_a, g_s = sim.step_backward(s_t, a_t, done, g_s_next, g_r,
                                     g_depth if ctx.has[0] else None,
                                     g_lidar if ctx.has[1] else None)
        return None, g_s, g_a
