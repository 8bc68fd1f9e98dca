"""The seeded input generators: trees, raw rate matrices, category rates, data."""
import numpy as np
import pytest
from scipy import integrate, stats

import synth
from synth.workloads import GTR_PAIRS, codon_frequencies_f3x4


def test_coalescent_root_height_and_shape():
    rng = np.random.default_rng(0)
    for n in (2, 3, 8, 100):
        h, p = synth.coalescent_tree(n, rng)
        assert h[2 * n - 2] == 1.0
        assert p[2 * n - 2] == -1 and (p[:-1] >= n).all()
        # binary: every internal node has two children, parents are older
        counts = np.bincount(p[:-1], minlength=2 * n - 1)
        assert (counts[n:] == 2).all() and (counts[:n] == 0).all()
        assert (h[p[:-1]] >= h[:-1]).all()
    th = rng.uniform(0, 0.2, 50)
    h, p = synth.coalescent_tree(50, rng, tip_heights=th)
    assert np.isclose(h.max(), 1.0) and h[:50].min() == 0.0
    assert (h[p[:-1]] >= h[:-1]).all()


def test_discrete_gamma_mean_method():
    for alpha in (0.2, 0.5, 1.0, 3.0):
        for C in (1, 2, 4, 8):
            r, w = synth.discrete_gamma(alpha, C)
            assert np.isclose((r * w).sum(), 1.0, atol=1e-12)
            assert np.all(np.diff(r) > 0) or C == 1
            # each rate is the conditional mean of its quantile bin
            g = stats.gamma(a=alpha, scale=1 / alpha)
            edges = np.concatenate([[0], g.ppf(np.arange(1, C) / C), [np.inf]])
            for c in range(C):
                m, _ = integrate.quad(lambda x: x * g.pdf(x), edges[c], edges[c + 1], limit=200)
                assert np.isclose(r[c], C * m, rtol=1e-6, atol=1e-9)
    r, _ = synth.discrete_gamma(1e4, 4)
    assert np.allclose(r, 1.0, atol=0.02)


def test_model_builders():
    pi = np.array([0.1, 0.2, 0.3, 0.4])
    Q, D = synth.hky_raw(3.0, pi)
    assert np.allclose(Q.sum(1), 0) and np.allclose(D.sum(1), 0)
    assert np.allclose(pi[:, None] * Q, (pi[:, None] * Q).T)
    assert np.isclose(Q[0, 2], 3.0 * pi[2]) and np.isclose(Q[0, 1], pi[1])
    Q2, _ = synth.hky_raw(3.0 + 1e-6, pi)
    assert np.allclose((Q2 - Q) / 1e-6, D, atol=1e-8)
    s = np.arange(1.0, 7.0)
    Q, dQ = synth.gtr_raw(s, pi)
    assert np.allclose(pi[:, None] * Q, (pi[:, None] * Q).T)
    for k, (i, j) in enumerate(GTR_PAIRS):
        assert np.isclose(Q[i, j], s[k] * pi[j])
        s2 = s.copy()
        s2[k] += 1.0
        assert np.allclose(synth.gtr_raw(s2, pi)[0] - Q, dQ[k])


def test_gy94_structure():
    rng = np.random.default_rng(1)
    pi = codon_frequencies_f3x4(rng)
    assert len(pi) == 61 and np.isclose(pi.sum(), 1.0)
    Q, Dk, Dw = synth.gy94_raw(2.0, 0.3, pi)
    assert Q.shape == (61, 61)
    assert np.allclose(Q.sum(1), 0)
    assert np.allclose(pi[:, None] * Q, (pi[:, None] * Q).T)
    # each codon has exactly 9 single-nucleotide neighbours minus stop codons
    nz = (Q > 0).sum(1)
    assert nz.max() <= 9 and nz.min() >= 5
    Q2, _, _ = synth.gy94_raw(2.0, 0.3 + 1e-6, pi)
    assert np.allclose((Q2 - Q) / 1e-6, Dw, atol=1e-7)
    Q3, _, _ = synth.gy94_raw(2.0 + 1e-6, 0.3, pi)
    assert np.allclose((Q3 - Q) / 1e-6, Dk, atol=1e-7)
    # TTT (Phe) -> TTC (Phe): synonymous transition
    a, b = synth.SENSE_CODONS.index(0), synth.SENSE_CODONS.index(1)
    assert np.isclose(Q[a, b], 2.0 * pi[b])


def test_simulated_frequencies_approach_pi():
    """Stationary process: tip state frequencies ~ pi (chi-square sanity)."""
    rng = np.random.default_rng(7)
    h, p = synth.coalescent_tree(30, rng)
    pi = np.array([0.1, 0.2, 0.3, 0.4])
    Q, _ = synth.hky_raw(4.0, pi)
    aln = synth.simulate_alignment(h * 5, p, [], np.zeros(1, np.int32), Q[None], pi, np.ones(1),
                                   4000, rng)
    counts = np.bincount(aln[0], minlength=4)
    chi2 = ((counts - 4000 * pi) ** 2 / (4000 * pi)).sum()
    assert chi2 < stats.chi2.ppf(0.999, 3)


def test_workload_shapes():
    w1 = synth.hky_8taxa()
    assert w1.n_taxa == 8 and w1.n_epochs == 2 and w1.pattern_weights.sum() == 200
    assert np.isclose(w1.boundaries[0], 0.5)
    w2 = synth.small_nucleotide(5, 20, 100)
    assert w2.n_categories == 4 and w2.n_epochs == 3
    assert ((w2.pattern_weights >= 1) & (w2.pattern_weights <= 20)).all()
    b = synth.asym50_forest(n_trees=3, taxa=(50, 60))
    assert len(b.trees) == 3 and all(t.K == 50 and t.reversible == 0 for t in b.trees)


def test_exchange_builder_and_new_shapes():
    rng = np.random.default_rng(4)
    pi = rng.dirichlet(np.ones(7))
    s = rng.lognormal(size=21)
    Q, dQ = synth.exchange_raw(s, pi)
    assert np.allclose(Q.sum(1), 0) and np.allclose(pi[:, None] * Q, (pi[:, None] * Q).T)
    for k in (0, 5, 20):
        s2 = s.copy()
        s2[k] += 1.0
        assert np.allclose(synth.exchange_raw(s2, pi)[0] - Q, dQ[k])
    f = synth.flu_seasonal()
    assert f.K == 7 and f.n_epochs == 13 and f.n_taxa == 522 and f.n_patterns == 1
    assert list(f.epoch_to_matrix) == [e % 2 for e in range(13)] and f.n_matrices == 2
    assert np.allclose(f.boundaries, np.arange(1, 13) / 13) and np.isclose(f.heights[-1], 1.0)
    assert f.n_params == 42 and f.heights[:522].min() == 0.0 and f.heights[:522].max() > 0.1
    a = synth.amino_acid(n_taxa=20, n_sites=50)
    assert a.K == 20 and a.n_epochs == 3 and a.pattern_weights.sum() == 50 and a.n_params == 9
