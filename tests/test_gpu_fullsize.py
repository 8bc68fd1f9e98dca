"""Parity at the full workload sizes (the launch configuration bench.py
times): the nucleotide GTR case (500 taxa, 10,000 patterns, 4 categories, 3
epochs) against the oracle outright; the codon GY94 case (128 taxa, 5,000
codon sites, 4 categories, 4 epochs) on a sample of per-pattern values the
oracle computes in seconds, and its gradient against central finite
differences of the FP64 GPU likelihood."""
import numpy as np
import pytest

import oracle
import synth
from paper_1309_3075_b300 import binding
from paper_1309_3075_b300.binding import (EPOCH_FP32, EPOCH_FP32_TC, EPOCH_FP32_TC_BF16, EPOCH_FP64,
                                          EpochLikelihood)
from tolerances import grad_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1309_3075_b300 import build

    build.build()


@pytest.fixture(scope="module")
def gtr_full():
    return synth.gtr_500taxa()


@pytest.fixture(scope="module")
def gy94_full():
    return synth.gy94_128taxa()


def maxrel(g, ref):
    return np.abs(np.asarray(g) - np.asarray(ref)).max() / max(np.abs(ref).max(), 1e-300)


@pytest.mark.parametrize("prec,tol", [(EPOCH_FP64, 1e-10), (EPOCH_FP32, 1e-5)])
def test_gtr_full_size_lnl_and_gradient(gtr_full, prec, tol):
    w = gtr_full
    lik = EpochLikelihood(w, precision=prec)
    try:
        lnl, g = lik.evaluate(with_gradient=True)
    finally:
        lik.close()
    ref = oracle.gradient(w)
    assert abs(lnl - ref["lnL"]) <= tol * abs(ref["lnL"])
    for key in ("heights", "boundaries", "params", "branch_rates"):
        ok, worst = grad_close(g[key], ref[key], prec)
        assert ok, (key, worst)


@pytest.mark.parametrize("prec,tol", [(EPOCH_FP64, 1e-10), (EPOCH_FP32, 1e-5),
                                      (EPOCH_FP32_TC, 1e-5), (EPOCH_FP32_TC_BF16, 1e-5)])
def test_gy94_full_size_sampled_sites(gy94_full, prec, tol):
    w = gy94_full
    lik = EpochLikelihood(w, precision=prec)
    try:
        lnl = lik.log_likelihood()
        site = lik.site_log_likelihoods()
    finally:
        lik.close()
    # lnL is the weighted sum of the per-pattern values
    assert abs(lnl - (w.pattern_weights * site).sum()) <= 1e-12 * abs(lnl)
    idx = np.random.default_rng(7).choice(w.n_patterns, size=160, replace=False)
    idx.sort()
    sub = w.replace(tips=np.ascontiguousarray(w.tips[:, idx]),
                    pattern_weights=w.pattern_weights[idx])
    _, rsite = oracle.log_likelihood(sub)
    # each sampled pattern on its own, at ten times the lnL bound
    assert np.all(np.abs(site[idx] - rsite) <= 10 * tol * np.abs(rsite)), \
        np.max(np.abs(site[idx] - rsite) / np.abs(rsite))


@pytest.fixture(scope="module")
def gy94_slice(gy94_full):
    """The codon gradient workload at its own shape (128 taxa, 4 epochs,
    C = 4, the shared kappa and the four omega_k) on 32 of its patterns, with
    the oracle's analytic gradient (its cost is per branch, about a minute)."""
    w = gy94_full.slice_patterns(0, 32)
    return w, oracle.gradient(w), oracle.log_likelihood(w)[1]


@pytest.mark.parametrize("prec", [EPOCH_FP64, EPOCH_FP32, EPOCH_FP32_TC, EPOCH_FP32_TC_BF16])
def test_gy94_gradient_against_oracle_at_config_shape(gy94_slice, prec):
    """d lnL / d (node heights, boundaries, kappa, omega_k) of the codon
    epoch model (Eq. convolution differentiated), GPU against the FP64 oracle
    element by element, and lnL per pattern, on every precision path."""
    w, ref, rsite = gy94_slice
    lik = EpochLikelihood(w, precision=prec)
    try:
        lnl, g = lik.evaluate(with_gradient=True)
        site = lik.site_log_likelihoods()
    finally:
        lik.close()
    ltol = 1e-10 if prec == EPOCH_FP64 else 1e-5
    assert abs(lnl - ref["lnL"]) <= ltol * abs(ref["lnL"]), (lnl, ref["lnL"])
    assert np.all(np.abs(site - rsite) <= 10 * ltol * np.abs(rsite))
    internal = np.arange(w.n_taxa, 2 * w.n_taxa - 1)
    internal = internal[w.parent[internal] >= 0]
    for key, idx in (("heights", internal), ("boundaries", slice(None)), ("params", slice(None))):
        got, want = np.asarray(g[key])[idx], np.asarray(ref[key])[idx]
        ok, worst = grad_close(got, want, prec)
        assert ok, (key, worst, got, want)


def test_gy94_full_size_gradient_vs_finite_differences(gy94_full):
    """Config: d lnL / d (node heights, boundaries, kappa, omega_k) by the
    adjoint kernels, against central differences (h = 1e-6) of the FP64 GPU
    lnL, on a sample of coordinates; the FP32 path's gradient against the
    FP64 one."""
    w = gy94_full
    lik = EpochLikelihood(w, precision=EPOCH_FP64)
    lik32 = EpochLikelihood(w, precision=EPOCH_FP32)
    liktc = EpochLikelihood(w, precision=EPOCH_FP32_TC)
    try:
        lnl, g = lik.evaluate(with_gradient=True)
        _, g32 = lik32.evaluate(with_gradient=True)
        lnltc, gtc = liktc.evaluate(with_gradient=True)

        def lnl_at(heights=None, bounds=None, Q=None):
            if Q is not None:
                binding.epoch_set_rate_matrices(lik.ctx, Q, w.pi)
            if bounds is not None:
                binding.epoch_set_boundaries(lik.ctx, bounds)
            if heights is not None:
                binding.epoch_set_heights(lik.ctx, heights)
            val = lik.evaluate(with_gradient=False)[0]
            binding.epoch_set_rate_matrices(lik.ctx, w.Q, w.pi)
            binding.epoch_set_boundaries(lik.ctx, w.boundaries)
            binding.epoch_set_heights(lik.ctx, w.heights)
            return val

        h = 1e-6
        rng = np.random.default_rng(3)
        nodes = rng.choice(np.arange(w.n_taxa, 2 * w.n_taxa - 2), size=4, replace=False)
        for u in nodes:
            hp, hm = w.heights.copy(), w.heights.copy()
            hp[u] += h
            hm[u] -= h
            fd = (lnl_at(heights=hp) - lnl_at(heights=hm)) / (2 * h)
            assert abs(g["heights"][u] - fd) <= 1e-4 * max(1.0, abs(fd)), (u, g["heights"][u], fd)
        for j in range(w.n_epochs - 1):
            bp, bm = w.boundaries.copy(), w.boundaries.copy()
            bp[j] += h
            bm[j] -= h
            fd = (lnl_at(bounds=bp) - lnl_at(bounds=bm)) / (2 * h)
            assert abs(g["boundaries"][j] - fd) <= 1e-4 * max(1.0, abs(fd)), (j, g["boundaries"][j], fd)
        # model parameters: the h = 1e-6 central difference of a lnL of
        # magnitude ~1e5 carries ~1e-3 of rounding noise (1e-14 relative
        # evaluation noise / h), so it is checked against its own noise
        # bound, and a fourth-order stencil at h = 1e-4 (truncation
        # O(h^4), noise ~1e-4) is held to 1e-4 relative
        noise = 1e-13 * abs(lnl) / h
        for a in range(w.n_params):
            fd = (lnl_at(Q=w.Q + h * w.dQ[a]) - lnl_at(Q=w.Q - h * w.dQ[a])) / (2 * h)
            assert abs(g["params"][a] - fd) <= 1e-4 * abs(fd) + noise, (w.param_names[a], g["params"][a], fd)
            H = 1e-4
            f = [lnl_at(Q=w.Q + k * H * w.dQ[a]) for k in (2, 1, -1, -2)]
            fd4 = (-f[0] + 8 * f[1] - 8 * f[2] + f[3]) / (12 * H)
            assert abs(g["params"][a] - fd4) <= 1e-4 * max(1.0, abs(fd4)), (w.param_names[a], g["params"][a], fd4)
        for k in ("heights", "boundaries", "params"):
            ok, worst = grad_close(g32[k], g[k], EPOCH_FP32)
            assert ok, (k, worst)
            ok, worst = grad_close(gtc[k], g[k], EPOCH_FP32_TC)
            assert ok, ("tensor cores", k, worst)
        assert abs(lnl - lik32.evaluate(with_gradient=False)[0]) <= 1e-5 * abs(lnl)
        assert abs(lnl - lnltc) <= 1e-5 * abs(lnl)
    finally:
        lik.close()
        lik32.close()
        liktc.close()


def test_forest_full_size_sampled_trees():
    """The 256-tree batch in the launch the bench times.  The oracle (dense
    uniformisation, a few seconds per 1,000-taxon tree at K = 50) checks the
    three smallest trees, the 13th smallest, the two largest and the largest
    tree with 8 epochs."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1309_3075_b300.binding import EpochBatch
    bw = synth.asym50_forest()
    b = EpochBatch(bw.trees)
    try:
        got = b.evaluate()
    finally:
        b.close()
    assert np.all(np.isfinite(got))
    sizes = np.array([t.n_taxa for t in bw.trees])
    order = np.argsort(sizes, kind="stable")
    pick = [int(order[i]) for i in (0, 1, 2, 12, -1, -2)]
    eight = [t for t in range(len(bw.trees)) if bw.trees[t].n_epochs == 8]
    pick.append(max(eight, key=lambda t: bw.trees[t].n_taxa))
    for t in pick:
        ref = oracle.log_likelihood(bw.trees[t])[0]
        assert abs(got[t] - ref) <= 1e-5 * abs(ref), (t, got[t], ref)


def test_forest_gradient_full_size_sampled_trees():
    """The batched lnL + gradient launch over all 256 trees; the oracle's
    gradient (a few seconds per 400-taxon tree at K = 50) checks the three
    smallest trees and the smallest tree with 8 epochs."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1309_3075_b300.binding import EpochBatch
    bw = synth.asym50_forest()
    b = EpochBatch(bw.trees)
    try:
        lnl, dh, db = b.evaluate_gradient()
    finally:
        b.close()
    assert np.all(np.isfinite(lnl))
    sizes = np.array([t.n_taxa for t in bw.trees])
    order = np.argsort(sizes, kind="stable")
    pick = [int(order[i]) for i in (0, 1, 2)]
    eight = [t for t in range(len(bw.trees)) if bw.trees[t].n_epochs == 8]
    pick.append(min(eight, key=lambda t: bw.trees[t].n_taxa))
    for t in pick:
        w = bw.trees[t]
        ref = oracle.gradient(w)
        assert abs(lnl[t] - ref["lnL"]) <= 1e-5 * abs(ref["lnL"]), (t, lnl[t], ref["lnL"])
        ok, worst = grad_close(dh[t], ref["heights"], EPOCH_FP32)
        assert ok, ("heights", t, worst)
        if w.n_epochs > 1:
            scale = max(np.abs(ref["boundaries"]).max(), np.abs(ref["heights"]).max())
            ok, worst = grad_close(db[t], ref["boundaries"], EPOCH_FP32, scale)
            assert ok, ("boundaries", t, worst)
