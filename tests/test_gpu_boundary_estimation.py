"""Estimating an epoch boundary from data with the library's gradient
(Discussion: transition times taken as known are a limitation; the boundary
derivative of the differentiated Eq. convolution makes them estimable).

Data are simulated under a two-epoch model whose processes differ strongly
(HKY with kappa 1 below the boundary and kappa 12 above it, shared pi), with
the boundary at b* = 0.35 of the root height.  From a perturbed start the
boundary is moved uphill along d lnL / d b, using only library calls
(epoch_set_boundaries, the evaluation and its gradient), with a step that
halves whenever lnL would decrease.  The estimate must lie near b*, the
gradient must vanish there, and the FP64 oracle (no shared code) must find
lnL at the estimate above lnL a small step to either side."""
import numpy as np
import pytest

import oracle
import synth
from paper_1309_3075_b300 import binding
from paper_1309_3075_b300.binding import EPOCH_FP32, EPOCH_FP64, EpochLikelihood

pytestmark = pytest.mark.gpu

B_TRUE = 0.35


@pytest.fixture(scope="module")
def two_epoch_data():
    rng = np.random.default_rng(4242)
    heights, parent = synth.coalescent_tree(96, rng)
    pi = np.array([0.3, 0.2, 0.2, 0.3])
    Q = np.stack([synth.hky_raw(1.0, pi)[0], synth.hky_raw(12.0, pi)[0]])
    b = np.array([B_TRUE])
    phi = np.arange(2, dtype=np.int32)
    aln = synth.simulate_alignment(heights, parent, b, phi, Q, pi, np.ones(1), 20000, rng)
    tips, w = synth.compress_patterns(aln)
    return synth.Workload("hky-kappa-switch-96taxa", 4, b, phi, Q, pi, np.ones(1), np.ones(1),
                          heights, parent, tips, w)


def _ascend(lik, w, b0, iters=60):
    """Gradient ascent on the boundary through the C ABI; returns the path."""
    def at(b):
        binding.epoch_set_boundaries(lik.ctx, np.array([b]))
        lnl, g = lik.evaluate(with_gradient=True)
        return lnl, float(g["boundaries"][0])

    b = b0
    lnl, g = at(b)
    step = 0.02 / max(abs(g), 1e-300)  # first move about 0.02 of the root height
    path = [(b, lnl, g)]
    for _ in range(iters):
        cand = float(np.clip(b + step * g, 0.02, 0.98))
        lc, gc = at(cand)
        if lc >= lnl:
            b, lnl, g = cand, lc, gc
            step *= 1.5
        else:
            step *= 0.5
        path.append((b, lnl, g))
        if abs(g) * step < 1e-7:
            break
    return path


@pytest.mark.parametrize("prec", [EPOCH_FP64, EPOCH_FP32])
@pytest.mark.parametrize("b0", [0.2, 0.55])
def test_boundary_recovered_by_gradient_ascent(two_epoch_data, prec, b0):
    w = two_epoch_data.replace(boundaries=np.array([b0]))
    lik = EpochLikelihood(w, precision=prec)
    try:
        path = _ascend(lik, w, b0)
        g0 = abs(path[0][2])
        b_hat, lnl_hat, g_hat = path[-1]
        binding.epoch_set_boundaries(lik.ctx, np.array([B_TRUE]))
        lnl_true = lik.evaluate(with_gradient=False)[0]
    finally:
        lik.close()
    assert abs(b_hat - B_TRUE) < 0.05, (b0, b_hat)
    # a stationary point (FP32 lnL carries ~1e-7 relative rounding, which
    # limits how finely its comparisons can place the maximum)
    assert abs(g_hat) <= (1e-3 if prec == EPOCH_FP64 else 1e-2) * g0, (g_hat, g0)
    assert lnl_hat >= lnl_true - 1e-6 * abs(lnl_true)  # at least as likely as the truth
    # the oracle, independently: lnL at the estimate above lnL 0.01 to either side
    ref = [oracle.log_likelihood(two_epoch_data.replace(boundaries=np.array([x])))[0]
           for x in (b_hat - 0.01, b_hat, b_hat + 0.01)]
    assert ref[1] > ref[0] and ref[1] > ref[2], ref
