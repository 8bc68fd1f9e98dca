"""Parity on the two further workload shapes, through the C ABI against the
FP64 oracle at full size:

* seasonal phylogeography shaped like the paper's influenza timing case
  (Results): 522 dated tips, K = 7 locations, 13 epochs alternating between
  two processes through the epoch-to-matrix map, one location trait; the
  symmetric model with the gradient in all 42 exchangeabilities, the
  asymmetric model with the height, boundary and branch-rate gradients, and
  64 replicate traits;
* amino-acid-shaped data: K = 20, 3 epochs, 200 taxa, 2,000 sites (also on
  the 32-wide tensor-core tiles).

Tolerances as in the other parity tests: lnL 1e-10 (FP64) and 1e-5 (FP32)
relative; gradients 1e-9 and 1e-4 relative per component (floors in
tests/tolerances.py); branch matrices 1e-12.
"""
import numpy as np
import pytest

import oracle
import synth
from paper_1309_3075_b300.binding import EPOCH_FP32, EPOCH_FP32_TC, EPOCH_FP64, EpochLikelihood
from tolerances import GRAD_TOL, LNL_TOL, grad_close

pytestmark = pytest.mark.gpu



@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1309_3075_b300 import build

    build.build()


def check(w, prec, params=True):
    lik = EpochLikelihood(w, precision=prec)
    try:
        lnl, g = lik.evaluate(with_gradient=True)
        site = lik.site_log_likelihoods()
    finally:
        lik.close()
    ref = oracle.gradient(w)
    rlnl, rsite = oracle.log_likelihood(w)
    assert abs(lnl - rlnl) <= LNL_TOL[prec] * abs(rlnl), (w.name, lnl, rlnl)
    assert np.allclose(site, rsite, rtol=10 * LNL_TOL[prec], atol=10 * LNL_TOL[prec] * np.abs(rsite).max())
    nn = 2 * w.n_taxa - 1
    ok, worst = grad_close(g["heights"], ref["heights"], prec)
    assert ok, ("heights", worst)
    scale = max(np.abs(ref["boundaries"]).max(), np.abs(ref["heights"]).max())
    ok, worst = grad_close(g["boundaries"], ref["boundaries"], prec, scale)
    assert ok, ("boundaries", worst)
    ok, worst = grad_close(g["branch_rates"][:nn], ref["branch_rates"], prec)
    assert ok, ("branch rates", worst)
    if params:
        ok, worst = grad_close(g["params"], ref["params"], prec)
        assert ok, ("params", worst)
    return g, ref


@pytest.fixture(scope="module")
def seasonal():
    return synth.flu_seasonal()


@pytest.mark.parametrize("prec", [EPOCH_FP64, EPOCH_FP32])
def test_seasonal_13_epochs_symmetric(seasonal, prec):
    check(seasonal, prec)


def test_seasonal_branch_matrices_across_many_boundaries(seasonal):
    """Branches that cross the most boundaries: the product of up to 13
    segment exponentials, against the oracle's product entry by entry."""
    w = seasonal
    lik = EpochLikelihood(w, precision=EPOCH_FP64)
    try:
        lik.log_likelihood()
        root = 2 * w.n_taxa - 2
        crossings = []
        for v in range(root):
            lo, hi = w.heights[v], w.heights[w.parent[v]]
            crossings.append(int(((w.boundaries > lo) & (w.boundaries < hi)).sum()))
        order = np.argsort(crossings)[::-1][:6]
        assert crossings[order[0]] >= 5
        for v in order:
            P = lik.branch_matrix(int(v), 0)
            assert np.allclose(P, oracle.branch_matrix(w, int(v), 0), rtol=0, atol=1e-12)
    finally:
        lik.close()


@pytest.mark.parametrize("prec", [EPOCH_FP64, EPOCH_FP32])
def test_seasonal_asymmetric(prec):
    w = synth.flu_seasonal(seed=1317, reversible=False)
    check(w, prec, params=False)


@pytest.mark.parametrize("prec", [EPOCH_FP64, EPOCH_FP32])
def test_seasonal_replicate_traits_three_processes(prec):
    w = synth.flu_seasonal(seed=1318, n_traits=64, n_processes=3, n_taxa=300)
    check(w, prec)


@pytest.mark.parametrize("prec", [EPOCH_FP64, EPOCH_FP32, EPOCH_FP32_TC])
def test_amino_acid_20_states(prec):
    check(synth.amino_acid(), prec)
