"""Batched trees (epoch_batch_*): one persistent launch over many uneven
trees with their own epochs and asymmetric rate matrices, through the C ABI,
against the FP64 oracle tree by tree (FP32 tolerance: 1e-5 relative lnL)
and against the single-tree entry points."""
import numpy as np
import pytest

import oracle
import synth

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
