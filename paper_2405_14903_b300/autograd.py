"""``torch.autograd.Function`` over a differentiable rollout (Sec. 2.3.4).

Forward: ``nf_set_params`` + ``nf_set_velocity`` (optionally projected) +
``nf_step`` x T + ``nf_loss``. Backward: ``nf_backward`` (checkpointed BPTT,
Sec. 2.3.2 and 2.3.3) returning dJ/dtheta and dJ/dU^0; the gradients are
derived analytically by the library, not by autograd tracing.
"""

from __future__ import annotations

import numpy as np
import torch

from .api import Episode


class RolloutLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, ux, uy, uz, episode: Episode, steps: int, loss: str,
                project: bool):
        episode.set_params(theta.detach().cpu().numpy().astype(np.float64))
        episode.set_velocity([ux.detach(), uy.detach(), uz.detach()], project=project)
        episode.step(steps)
        J, gU = episode.loss(loss, want_grad=True, dtype=ux.dtype)
        ctx.episode = episode
        ctx.gU = gU
        ctx.theta_device = theta.device
        return torch.tensor(J, dtype=torch.float64, device=theta.device)

    @staticmethod
    def backward(ctx, gJ):
        ep: Episode = ctx.episode
        gth, gU0, _ = ep.backward(ctx.gU, want_gU0=True)
        s = float(gJ)
        gth_t = torch.tensor(gth * s, dtype=torch.float64, device=ctx.theta_device)
        return (gth_t, gU0[0] * s, gU0[1] * s, gU0[2] * s, None, None, None, None)


def rollout_loss(episode: Episode, theta, u0, steps, loss="kinetic_energy", project=True):
    """J(theta, u0) of a T-step rollout, differentiable w.r.t. theta and u0."""
    return RolloutLoss.apply(theta, u0[0], u0[1], u0[2], episode, steps, loss, project)
