"""torch.autograd.Function around the libepoch likelihood and its adjoint.

Forward runs the whole path (branch matrices, pruning, root) on the device;
backward returns the gradient that the same evaluation produced with the
pre-order adjoint pass (no finite differences, no CPU arithmetic).  Torch is
used for the tensors only.
"""
from __future__ import annotations

import numpy as np
import torch

from paper_1309_3075_b300.binding import (
    EpochLikelihood,
    epoch_set_boundaries,
    epoch_set_heights,
    epoch_set_rate_derivatives,
    epoch_set_rate_matrices,
)


class EpochLogLikelihood(torch.autograd.Function):
    """lnL(heights, boundaries, theta).

    ``lik`` is an EpochLikelihood whose tips, categories and topology are
    set; ``model_fn(theta) -> (Q [S][K][K], dQ [n][S][K][K])`` gives the raw
    rate matrices and their derivatives for parameter values theta (for
    example an HKY or GY94 builder); ``pi``, ``normalise`` and ``reversible``
    are passed through to epoch_set_rate_matrices.
    """

    @staticmethod
    def forward(ctx, lik: EpochLikelihood, model_fn, pi, heights, boundaries, theta,
                normalise=1, reversible=1):
        th = theta.detach().cpu().numpy().astype(np.float64)
        Q, dQ = model_fn(th)
        epoch_set_rate_matrices(lik.ctx, Q, pi, normalise, reversible)
        epoch_set_rate_derivatives(lik.ctx, dQ)
        lik.n_params = 0 if dQ is None else int(np.asarray(dQ).shape[0])
        if lik.E > 1:
            epoch_set_boundaries(lik.ctx, boundaries.detach().cpu().numpy().astype(np.float64))
        epoch_set_heights(lik.ctx, heights.detach().cpu().numpy().astype(np.float64))
        want = any(t.requires_grad for t in (heights, boundaries, theta))
        lnl, g = lik.evaluate(with_gradient=want)
        if want:
            ctx.save_for_backward(torch.from_numpy(g["heights"]), torch.from_numpy(g["boundaries"]),
                                  torch.from_numpy(g["params"]))
        ctx.shapes = (heights.device, boundaries.device, theta.device)
        return torch.tensor(lnl, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_out):
        gh, gb, gp = ctx.saved_tensors
        dh, db, dt = ctx.shapes
        go = grad_out.detach().cpu().to(torch.float64)
        return (None, None, None, (go * gh).to(dh), (go * gb).to(db), (go * gp).to(dt), None,
                None)


def log_likelihood(lik, model_fn, pi, heights, boundaries, theta, normalise=1, reversible=1):
    return EpochLogLikelihood.apply(lik, model_fn, pi, heights, boundaries, theta, normalise,
                                    reversible)
