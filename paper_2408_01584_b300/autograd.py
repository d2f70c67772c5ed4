"""torch.autograd.Function over the differentiable rollout of the C ABI.

    ell = rollout_objective(env, actions, obs_weight, reward_weight, state0)

runs gd_rollout_objective (forward, checkpointing every ckpt_every steps)
and, on backward, gd_rollout_backward (recompute + adjoint kernels).  Only
argument marshalling happens here.  The env must be created with
GD_DIFFERENTIABLE; the backward of one call must run before the env's next
objective rollout, and `actions` must not be modified in between.
"""
from __future__ import annotations

import torch

from . import gd


class RolloutObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, actions, state0, env, obs_weight, reward_weight):
        T, A = actions.shape[0], actions.shape[1]
        actions = actions.detach().contiguous()
        gd.gd_reset(env.h, None)
        if state0 is not None:
            gd.gd_set_state(env.h, state0.detach().contiguous())
        ell = torch.empty(T, A, dtype=torch.float32, device=actions.device)
        gd.gd_rollout_objective(env.h, T, actions, obs_weight, reward_weight, ell, env.obs)
        ctx.env, ctx.actions, ctx.w, ctx.wr = env, actions, obs_weight, float(reward_weight)
        ctx.has_state0 = state0 is not None
        return ell

    @staticmethod
    def backward(ctx, d_ell):
        env, actions = ctx.env, ctx.actions
        d_actions = torch.empty_like(actions)
        d_state0 = torch.empty(actions.shape[1], 4, dtype=torch.float32, device=actions.device)
        gd.gd_rollout_backward(env.h, ctx.w, ctx.wr, d_ell.contiguous(), d_actions, d_state0)
        return d_actions, (d_state0 if ctx.has_state0 else None), None, None, None


def rollout_objective(env, actions, obs_weight, reward_weight=1.0, state0=None):
    """Per-step, per-agent objective terms ell [T, A] of a rollout from the
    env's initial snapshot (or from state0 [A, 4]), differentiable w.r.t.
    actions [T, A, 2] and state0."""
    return RolloutObjective.apply(actions, state0, env, obs_weight, reward_weight)
