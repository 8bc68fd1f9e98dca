"""Outputs built on the adjoint pass, through the C ABI against the FP64
oracle, on the FP64 path and on the FP32 paths (K = 4 level kernels, the
few-pattern kernels at K = 7, generic kernels, the tensor-core kernels at
K = 61):

* expected transition counts (Markov jumps) per branch and per epoch;
  tolerances 1e-9 (FP64) and 1e-4 (FP32) relative to the largest count, the
  bounds of the gradient tests (the counts are contractions of the same G);
* marginal posterior state probabilities of every internal node; absolute
  tolerances 1e-10 (FP64) and 1e-5 (FP32) per probability."""
import numpy as np
import pytest

import oracle
import synth
from paper_1309_3075_b300 import binding
from paper_1309_3075_b300.binding import (EPOCH_FP32, EPOCH_FP32_TC, EPOCH_FP64, EpochError,
                                          EpochLikelihood)

pytestmark = pytest.mark.gpu

TOL = {EPOCH_FP64: 1e-9, EPOCH_FP32: 1e-4, EPOCH_FP32_TC: 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1309_3075_b300 import build

    build.build()


def check_counts(w, prec):
    lik = EpochLikelihood(w, precision=prec)
    try:
        lik.evaluate(with_gradient=True)
        pb, pe = lik.expected_counts()
    finally:
        lik.close()
    rb, re = oracle.expected_counts(w)
    scale = max(np.abs(rb).max(), 1e-300)
    assert np.abs(pb - rb).max() <= TOL[prec] * scale, (w.name, np.abs(pb - rb).max(), scale)
    assert np.abs(pe - re).max() <= TOL[prec] * max(np.abs(re).max(), 1e-300)
    return pb, pe


@pytest.mark.parametrize("prec", [EPOCH_FP64, EPOCH_FP32])
def test_counts_nucleotide_dated_rates(prec):
    w = synth.small_nucleotide(411, n_taxa=24, n_sites=150, n_cat=3, n_epochs=3, dated=True)
    w = w.replace(branch_rates=np.random.default_rng(4).uniform(0.6, 1.4, 2 * w.n_taxa - 1))
    check_counts(w, prec)


@pytest.mark.parametrize("prec", [EPOCH_FP64, EPOCH_FP32])
def test_counts_seasonal_trait(prec):
    """One location trait, 13 alternating epochs: the per-epoch counts are
    the paper's per-season summaries of location changes."""
    w = synth.flu_seasonal(seed=1319, n_taxa=60)
    pb, pe = check_counts(w, prec)
    assert pe.shape == (13, 7, 7)


def test_counts_codon_tensor_cores():
    w = synth.small_codon(412, n_taxa=10, n_sites=60, n_cat=2, n_epochs=2)
    check_counts(w, EPOCH_FP32_TC)


def test_counts_need_a_gradient_and_a_reversible_model():
    w = synth.tiny_tree_workload(413, K=4, n_taxa=6, n_sites=5, n_epochs=2)
    lik = EpochLikelihood(w, precision=EPOCH_FP64)
    try:
        lik.log_likelihood()
        with pytest.raises(EpochError) as e:
            lik.expected_counts()
        assert e.value.status == 2  # EPOCH_ERR_ORDER: no gradient of these inputs yet
        lik.evaluate(with_gradient=True)
        lik.expected_counts()
        binding.epoch_set_heights(lik.ctx, w.heights)  # new inputs: stale G
        with pytest.raises(EpochError) as e:
            lik.expected_counts()
        assert e.value.status == 2
    finally:
        lik.close()
    wa = synth.tiny_tree_workload(414, K=5, n_taxa=6, n_sites=5, n_epochs=2, reversible=False)
    lik = EpochLikelihood(wa, precision=EPOCH_FP64)
    try:
        lik.evaluate(with_gradient=True)
        with pytest.raises(EpochError) as e:
            lik.expected_counts()
        assert e.value.status == 7  # EPOCH_ERR_UNSUPPORTED
    finally:
        lik.close()


ANC_TOL = {EPOCH_FP64: 1e-10, EPOCH_FP32: 1e-5, EPOCH_FP32_TC: 1e-5}


@pytest.mark.parametrize("prec,make", [
    (EPOCH_FP64, lambda: synth.small_nucleotide(421, n_taxa=20, n_sites=90, n_cat=2, n_epochs=3)),
    (EPOCH_FP32, lambda: synth.small_nucleotide(421, n_taxa=20, n_sites=90, n_cat=2, n_epochs=3)),
    (EPOCH_FP32, lambda: synth.flu_seasonal(seed=1320, n_taxa=50, n_traits=3)),
    (EPOCH_FP32, lambda: synth.tiny_tree_workload(422, K=12, n_taxa=15, n_sites=300, n_epochs=3,
                                                  n_cat=2, reversible=False, missing_frac=0.1)),
    (EPOCH_FP32_TC, lambda: synth.small_codon(423, n_taxa=9, n_sites=80, n_cat=2, n_epochs=2)),
])
def test_ancestral_states_match_oracle(prec, make):
    """Posterior state probabilities of every internal node and pattern on
    the FP64 path, the K = 4 level kernels (cherries from their code-pair
    tables), the few-pattern kernels, the generic FP32 kernels (asymmetric
    model) and the tensor-core kernels; absolute error per probability."""
    w = make()
    lik = EpochLikelihood(w, precision=prec)
    try:
        lik.evaluate(with_gradient=True)
        got = lik.ancestral_states()
    finally:
        lik.close()
    ref = oracle.ancestral_states(w)
    assert got.shape == ref.shape
    assert np.abs(got - ref).max() <= ANC_TOL[prec], (w.name, np.abs(got - ref).max())
    assert np.allclose(got.sum(-1), 1.0, atol=1e-12)


@pytest.mark.parametrize("prec", [EPOCH_FP64, EPOCH_FP32])
def test_two_taxa_and_single_epoch_edges(prec):
    """Two taxa (the root is the only internal node, on the K = 4 path the
    root's own level) and a single epoch: ancestral states of the root and
    counts on both branches against the oracle."""
    w = synth.tiny_tree_workload(431, K=4, n_taxa=2, n_sites=9, n_epochs=1, n_cat=2, dated=True)
    lik = EpochLikelihood(w, precision=prec)
    try:
        lik.evaluate(with_gradient=True)
        anc = lik.ancestral_states()
        pb, pe = lik.expected_counts()
    finally:
        lik.close()
    assert anc.shape == (1, w.n_patterns, 4) and pe.shape == (1, 4, 4)
    assert np.abs(anc - oracle.ancestral_states(w)).max() <= ANC_TOL[prec]
    rb, re = oracle.expected_counts(w)
    assert np.abs(pb - rb).max() <= TOL[prec] * max(np.abs(rb).max(), 1e-300)
    assert np.abs(pe - re).max() <= TOL[prec] * max(np.abs(re).max(), 1e-300)


def test_tensor_core_request_with_many_categories_uses_simt():
    """EPOCH_FP32_TC with more categories than the tensor-core kernels take
    (C = 6 > 4) runs the SIMT kernels; results match the oracle."""
    w = synth.tiny_tree_workload(432, K=20, n_taxa=10, n_sites=150, n_epochs=2, n_cat=6)
    lik = EpochLikelihood(w, precision=EPOCH_FP32_TC)
    try:
        lnl, g = lik.evaluate(with_gradient=True)
    finally:
        lik.close()
    ref = oracle.gradient(w)
    assert abs(lnl - ref["lnL"]) <= 1e-5 * abs(ref["lnL"])
    assert np.abs(g["heights"] - ref["heights"]).max() <= 1e-4 * max(np.abs(ref["heights"]).max(), 1.0)
