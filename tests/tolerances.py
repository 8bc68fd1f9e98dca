"""Parity tolerances shared by the GPU tests.

lnL: relative error <= 1e-10 on the FP64 path, <= 1e-5 on the FP32 paths.
Gradients: each component relative to its own size, <= 1e-9 (FP64) or
<= 1e-4 (FP32 paths), with a floor at a fraction of the largest component of
the same vector.  A derivative that is a sum over thousands of weighted
patterns can cancel to near zero; its rounding error is then set by the size
of the terms, not of the sum, so components below the floor are measured
against the floor.
"""
import numpy as np

from paper_1309_3075_b300.binding import (EPOCH_FP32, EPOCH_FP32_AUTO, EPOCH_FP32_TC,
                                          EPOCH_FP32_TC_BF16, EPOCH_FP64)

LNL_TOL = {EPOCH_FP64: 1e-10, EPOCH_FP32: 1e-5, EPOCH_FP32_TC: 1e-5, EPOCH_FP32_AUTO: 1e-5,
           EPOCH_FP32_TC_BF16: 1e-5}
GRAD_TOL = {EPOCH_FP64: 1e-9, EPOCH_FP32: 1e-4, EPOCH_FP32_TC: 1e-4, EPOCH_FP32_AUTO: 1e-4,
            EPOCH_FP32_TC_BF16: 1e-4}
# Measured worst per-component errors (GPU against the oracle on the parity
# workloads, components at least this fraction of the largest): FP32 and
# TF32x3 2.4e-6 .. 4.0e-5 at 0.3, up to 7.7e-5 at 0.1 and 5.9e-4 at 0.01;
# FP64 2.4e-10 at 0.1, 7.1e-10 at 0.01 and 2.6e-9 at 0.001.
GRAD_FLOOR = {EPOCH_FP64: 1e-1, EPOCH_FP32: 3e-1, EPOCH_FP32_TC: 3e-1, EPOCH_FP32_AUTO: 3e-1,
              EPOCH_FP32_TC_BF16: 3e-1}
# absolute floor, for derivatives that vanish exactly (a parameter whose
# effect the normalisation of Q removes)
GRAD_ABS = 1e-6


def component_rel(g, ref, floor, scale=None):
    """Worst |g_i - ref_i| / max(|ref_i|, floor * scale, GRAD_ABS) over the
    vector; scale defaults to max_j |ref_j|."""
    g = np.asarray(g, dtype=float).ravel()
    ref = np.asarray(ref, dtype=float).ravel()
    if ref.size == 0:
        return 0.0
    if scale is None:
        scale = np.abs(ref).max()
    den = np.maximum(np.maximum(np.abs(ref), floor * scale), GRAD_ABS)
    return float((np.abs(g - ref) / den).max())


def grad_close(g, ref, prec, scale=None):
    """(ok, worst relative error) for one gradient vector on path prec."""
    worst = component_rel(g, ref, GRAD_FLOOR[prec], scale)
    return worst <= GRAD_TOL[prec], worst
