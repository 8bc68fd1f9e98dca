"""torch.autograd.Function around the libepoch likelihood and its adjoint.

Forward runs the whole path (branch matrices, pruning, root) on the device;
backward returns the gradient that the same evaluation produced with the
pre-order adjoint pass (no finite differences, no CPU arithmetic).  Torch is
used for the tensors only.

When the node heights are a CUDA tensor and the likelihood was created on a
known stream (``EpochLikelihood(..., cuda_stream=...)``), heights go to the
library and lnL and the gradient come back as device pointers
(epoch_set_heights_device, epoch_read_results_device): nothing of the
evaluation crosses to the host, and torch's stream is ordered after the
library's with an event.  Otherwise the host entry points are used.
"""
from __future__ import annotations

import numpy as np
import torch

from paper_1309_3075_b300.binding import (
    EpochLikelihood,
    epoch_evaluate_async,
    epoch_read_results_device,
    epoch_set_boundaries,
    epoch_set_heights,
    epoch_set_heights_device,
    epoch_set_rate_derivatives,
    epoch_set_rate_matrices,
)


def _split(g, nn, E, n_params):
    """Gradient vector layout of the library: heights, boundaries, parameters, rates."""
    return g[:nn], g[nn:nn + E - 1], g[nn + E - 1:nn + E - 1 + n_params]


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
        want = any(t.requires_grad for t in (heights, boundaries, theta))
        nn = 2 * lik.N - 1
        if heights.is_cuda and lik.cuda_stream:
            lib = torch.cuda.ExternalStream(lik.cuda_stream, device=heights.device)
            cur = torch.cuda.current_stream(heights.device)
            h = heights.detach().to(torch.float64).contiguous()
            lib.wait_stream(cur)  # h is written
            h.record_stream(lib)
            epoch_set_heights_device(lik.ctx, h.data_ptr())
            epoch_evaluate_async(lik.ctx, 1 if want else 0)
            out = torch.empty(1 + 2 * nn + (lik.E - 1) + lik.n_params, dtype=torch.float64,
                              device=heights.device)
            out.record_stream(lib)
            epoch_read_results_device(lik.ctx, out.data_ptr(),
                                      out[1:].data_ptr() if want else 0)
            cur.wait_stream(lib)
            lnl, g = out[0], out[1:]
            if want:
                gh, gb, gp = _split(g, nn, lik.E, lik.n_params)
                ctx.save_for_backward(gh, gb, gp)
        else:
            epoch_set_heights(lik.ctx, heights.detach().cpu().numpy().astype(np.float64))
            val, gd = lik.evaluate(with_gradient=want)
            lnl = torch.tensor(val, dtype=torch.float64)
            if want:
                ctx.save_for_backward(torch.from_numpy(gd["heights"]),
                                      torch.from_numpy(gd["boundaries"]),
                                      torch.from_numpy(gd["params"]))
        ctx.devices = (heights.device, boundaries.device, theta.device)
        return lnl

    @staticmethod
    def backward(ctx, grad_out):
        gh, gb, gp = ctx.saved_tensors
        dh, db, dt = ctx.devices
        go = grad_out.detach().to(torch.float64)
        return (None, None, None, (go.to(gh.device) * gh).to(dh), (go.to(gb.device) * gb).to(db),
                (go.to(gp.device) * gp).to(dt), None, None)


def log_likelihood(lik, model_fn, pi, heights, boundaries, theta, normalise=1, reversible=1):
    return EpochLogLikelihood.apply(lik, model_fn, pi, heights, boundaries, theta, normalise,
                                    reversible)
