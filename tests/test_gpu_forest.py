"""Batched trees (epoch_batch_*): one persistent launch over many uneven
trees with their own epochs and asymmetric rate matrices, through the C ABI,
against the FP64 oracle tree by tree (FP32 tolerance: 1e-5 relative lnL;
gradients per component as in tests/tolerances.py) and against the
single-tree entry points."""
import numpy as np
import pytest

import oracle
import synth
from tolerances import grad_close

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return torch


def test_forest_matches_oracle_tree_by_tree(cuda):
    from paper_1309_3075_b300.binding import EpochBatch
    bw = synth.asym50_forest(seed=2024, n_trees=12, K=50, taxa=(5, 40), epochs=(1, 8),
                             patterns=(1, 4))
    b = EpochBatch(bw.trees)
    try:
        got = b.evaluate()
        for t, w in enumerate(bw.trees):
            ref = oracle.log_likelihood(w)[0]
            assert abs(got[t] - ref) <= TOL * abs(ref), (t, got[t], ref)
        again = b.evaluate()  # graph replay: same launch, same order of sums
        assert np.array_equal(got, again)
        warps, ctas = b.launch_shape()
        assert warps in (4, 8) and ctas >= 1
    finally:
        b.close()


def test_forest_small_K_dated_tips_missing_data(cuda):
    from paper_1309_3075_b300.binding import EpochBatch
    trees = [synth.tiny_tree_workload(300 + i, K=k, n_taxa=n, n_sites=3, n_epochs=e, n_cat=1,
                                      reversible=False, dated=True, missing_frac=0.2)
             for i, (k, n, e) in enumerate([(6, 9, 3), (6, 2, 1), (6, 17, 4), (6, 33, 2)])]
    b = EpochBatch(trees)
    try:
        got = b.evaluate()
    finally:
        b.close()
    for t, w in enumerate(trees):
        ref = oracle.log_likelihood(w)[0]
        assert abs(got[t] - ref) <= TOL * abs(ref), (t, got[t], ref)


def _longest_mu_segment(w):
    """Largest mu * dt over the segments of w (mu = max_i |q_ii| of the
    normalised matrix of the segment's epoch): the length of the longest
    uniformisation series the batched kernel would run without splitting."""
    E = w.n_epochs
    mus = []
    for e in range(E):
        q = w.Q[w.epoch_to_matrix[e]]
        c = -(w.pi * np.diag(q)).sum() if w.normalise else 1.0
        mus.append(np.max(-np.diag(q)) / c)
    b = np.r_[w.boundaries, np.inf]
    best = 0.0
    for v, u in enumerate(w.parent):
        if u < 0:
            continue
        lo, hi = w.heights[v], w.heights[u]
        e = int(np.searchsorted(w.boundaries, lo, side="right"))
        while lo < hi:
            top = min(b[e], hi)
            best = max(best, mus[e] * (top - lo))
            lo, e = top, e + 1
    return best


@pytest.mark.parametrize("target", [50.0, 120.0, 400.0])
def test_forest_long_segments(cuda, target):
    """Branches far longer than the uniformisation rate's time scale: each
    tree is stretched so that its longest segment has mu dt = target.  Above
    mu dt ~ 88 the first Poisson weight exp(-mu dt) underflows in FP32, so the
    kernel must split such segments (exp(t Q) = exp(t Q / n)^n, Eq. convolution
    applied to equal pieces)."""
    from paper_1309_3075_b300.binding import EpochBatch
    for K, shapes in ((6, [(12, 1), (2, 1), (30, 4)]), (50, [(20, 2), (40, 3)])):
        trees = []  # one state count per batch
        for i, (n, e) in enumerate(shapes):
            w = synth.tiny_tree_workload(500 + 10 * i + K, K=K, n_taxa=n, n_sites=3, n_epochs=e,
                                         n_cat=1, reversible=False, dated=True, missing_frac=0.1)
            f = target / _longest_mu_segment(w)
            w = w.replace(heights=w.heights * f, boundaries=w.boundaries * f)
            assert np.isclose(_longest_mu_segment(w), target)
            trees.append(w)
        b = EpochBatch(trees)
        try:
            got = b.evaluate()
        finally:
            b.close()
        for t, w in enumerate(trees):
            ref = oracle.log_likelihood(w)[0]
            assert np.isfinite(got[t]), (K, t, got[t])
            assert abs(got[t] - ref) <= TOL * abs(ref), (K, t, got[t], ref)


def test_forest_of_one_equals_single_tree_path(cuda):
    from paper_1309_3075_b300.binding import EPOCH_FP32, EpochBatch, EpochLikelihood
    w = synth.tiny_tree_workload(77, K=12, n_taxa=60, n_sites=4, n_epochs=5, n_cat=1,
                                 reversible=False, dated=True)
    lik = EpochLikelihood(w, precision=EPOCH_FP32)
    try:
        single = lik.log_likelihood()
    finally:
        lik.close()
    b = EpochBatch([w])
    try:
        batch = b.evaluate()[0]
    finally:
        b.close()
    assert abs(batch - single) <= 1e-5 * abs(single)


def test_forest_status_codes(cuda):
    from paper_1309_3075_b300 import binding
    from paper_1309_3075_b300.binding import EpochError
    with pytest.raises(EpochError) as e:
        binding.epoch_batch_create(4, [5], [1], [5])  # more than 4 patterns
    assert e.value.status == 1
    b = binding.epoch_batch_create(4, [3, 4], [1, 2], [1, 2])
    try:
        with pytest.raises(EpochError) as e:
            binding.epoch_batch_evaluate_async(b)  # nothing set yet
        assert e.value.status == 2
        with pytest.raises(EpochError) as e:
            binding.epoch_batch_set_tip_data(b, np.full(3 + 8, 9), np.ones(3))  # code > K
        assert e.value.status == 1
    finally:
        binding.epoch_batch_destroy(b)


def _gradient_trees(K):
    """Uneven trees with dated tips, missing data, 1-6 epochs, a two-taxon
    tree and one stretched so that its longest segment has mu dt = 120."""
    shapes = [(9, 3), (2, 1), (17, 4), (33, 2), (24, 6), (12, 1)]
    trees = [synth.tiny_tree_workload(700 + 7 * i + K, K=K, n_taxa=n, n_sites=3, n_epochs=e,
                                      n_cat=1, reversible=False, dated=True, missing_frac=0.1)
             for i, (n, e) in enumerate(shapes)]
    w = trees[-1]
    f = 120.0 / _longest_mu_segment(w)
    trees[-1] = w.replace(heights=w.heights * f, boundaries=w.boundaries * f)
    return trees


@pytest.mark.parametrize("K", [6, 50])
def test_forest_gradient_matches_oracle_tree_by_tree(cuda, K):
    """d lnL_t / d (node heights, boundaries) of every tree from the batched
    pre-order adjoint (Eq. convolution differentiated segment by segment),
    against the oracle's analytic gradient; replays are bitwise equal, and the
    lnL of the gradient launch equals that of the likelihood launch."""
    from paper_1309_3075_b300.binding import EPOCH_FP32, EpochBatch
    trees = _gradient_trees(K)
    b = EpochBatch(trees)
    try:
        lnl, dh, db = b.evaluate_gradient()
        lnl2, dh2, db2 = b.evaluate_gradient()
        plain = b.evaluate()
    finally:
        b.close()
    for t, w in enumerate(trees):
        ref = oracle.gradient(w)
        assert abs(lnl[t] - ref["lnL"]) <= TOL * abs(ref["lnL"]), (t, lnl[t], ref["lnL"])
        assert abs(lnl[t] - plain[t]) <= 1e-12 * abs(plain[t])
        ok, worst = grad_close(dh[t], ref["heights"], EPOCH_FP32)
        assert ok, ("heights", t, worst, dh[t], ref["heights"])
        if w.n_epochs > 1:
            scale = max(np.abs(ref["boundaries"]).max(), np.abs(ref["heights"]).max())
            ok, worst = grad_close(db[t], ref["boundaries"], EPOCH_FP32, scale)
            assert ok, ("boundaries", t, worst, db[t], ref["boundaries"])
        else:
            assert db[t].size == 0
        assert np.array_equal(dh[t], dh2[t]) and np.array_equal(db[t], db2[t])


def test_forest_gradient_needs_a_gradient_evaluation(cuda):
    from paper_1309_3075_b300 import binding
    from paper_1309_3075_b300.binding import EpochBatch, EpochError
    trees = _gradient_trees(6)[:2]
    b = EpochBatch(trees)
    try:
        b.evaluate()
        with pytest.raises(EpochError) as e:
            binding.epoch_batch_read_gradient(b.b, 2, sum(2 * w.n_taxa - 1 for w in trees),
                                              sum(w.n_epochs - 1 for w in trees))
        assert e.value.status == 2
        b.evaluate_gradient()
        b.load(trees)  # new inputs: the gradient must be evaluated again
        with pytest.raises(EpochError) as e:
            binding.epoch_batch_read_gradient(b.b, 2, sum(2 * w.n_taxa - 1 for w in trees),
                                              sum(w.n_epochs - 1 for w in trees))
        assert e.value.status == 2
    finally:
        b.close()
