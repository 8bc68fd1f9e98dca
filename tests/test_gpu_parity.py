"""GPU parity: libepoch (through the C ABI) against the FP64 CPU oracle on the
same seeded inputs.

Tolerances: lnL relative error <= 1e-10 on the FP64 path and <= 1e-5 on
the FP32 paths.  Branch matrices on every path are FP64 and must match to
1e-12.  Gradients: FP64 path within 1e-9 of the oracle's, FP32 paths
within 1e-4, each component relative to its own size (floors in
tests/tolerances.py); 1e-4 is also the bound of the finite-difference check
of the gradient.
"""
import numpy as np
import pytest

import oracle
import synth
from paper_1309_3075_b300 import binding
from paper_1309_3075_b300.binding import (EPOCH_FP32, EPOCH_FP32_AUTO, EPOCH_FP32_TC,
                                          EPOCH_FP32_TC_BF16, EPOCH_FP64, EpochError,
                                          EpochLikelihood)
from tolerances import GRAD_TOL, LNL_TOL, grad_close

pytestmark = pytest.mark.gpu

@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1309_3075_b300 import build

    build.build()


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def check_lnl(w, prec, site_sample=None):
    lik = EpochLikelihood(w, precision=prec)
    try:
        lnl = lik.log_likelihood()
        site = lik.site_log_likelihoods()
    finally:
        lik.close()
    ref, rsite = oracle.log_likelihood(w)
    assert rel(lnl, ref) <= LNL_TOL[prec], (w.name, prec, lnl, ref, rel(lnl, ref))
    tol = LNL_TOL[prec] * 10
    assert np.allclose(site, rsite, rtol=tol, atol=tol * np.abs(rsite).max())
    return lnl


def check_grad(w, prec):
    lik = EpochLikelihood(w, precision=prec)
    try:
        lik.log_likelihood()
        g = lik.gradient()
    finally:
        lik.close()
    ref = oracle.gradient(w)
    nn = 2 * w.n_taxa - 1
    ok, worst = grad_close(g["heights"], ref["heights"], prec)
    assert ok, ("heights", worst)
    if w.n_epochs > 1:
        # a boundary derivative is a difference of per-segment terms of the
        # size of the height derivatives; it can cancel to ~0 (identical
        # processes on both sides), so its floor is on that scale
        scale = max(np.abs(ref["boundaries"]).max(), np.abs(ref["heights"]).max())
        ok, worst = grad_close(g["boundaries"], ref["boundaries"], prec, scale)
        assert ok, ("boundaries", worst, g["boundaries"], ref["boundaries"])
    ok, worst = grad_close(g["branch_rates"][:nn], ref["branch_rates"], prec)
    assert ok, ("branch rates", worst)
    if w.n_params and w.reversible:
        ok, worst = grad_close(g["params"], ref["params"], prec)
        assert ok, ("params", worst, g["params"], ref["params"])
    return g, ref


# ---------------------------------------------------------------------------
# likelihood
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("prec", [EPOCH_FP64, EPOCH_FP32])
def test_hky_8taxa_two_epochs(prec):
    w = synth.hky_8taxa()
    check_lnl(w, prec)
    check_grad(w, prec)


@pytest.mark.parametrize("prec", [EPOCH_FP64, EPOCH_FP32])
@pytest.mark.parametrize("dated", [False, True])
def test_nucleotide_several_tiles_ragged(prec, dated):
    # 700 patterns = two full 256-pattern tiles and a ragged tail
    w = synth.small_nucleotide(201, n_taxa=40, n_sites=700, n_cat=4, n_epochs=3, dated=dated)
    check_lnl(w, prec)
    check_grad(w, prec)


@pytest.mark.parametrize("prec", [EPOCH_FP64, EPOCH_FP32])
def test_branch_matrices_match_oracle(prec):
    w = synth.small_nucleotide(202, n_taxa=25, n_sites=50, n_cat=3, n_epochs=4, dated=True)
    lik = EpochLikelihood(w, precision=prec)
    try:
        lik.log_likelihood()
        for v in range(2 * w.n_taxa - 2):
            for c in range(w.n_categories):
                P = lik.branch_matrix(v, c)
                assert np.allclose(P, oracle.branch_matrix(w, v, c), rtol=0, atol=1e-12)
    finally:
        lik.close()


@pytest.mark.parametrize("prec", [EPOCH_FP32, EPOCH_FP32_TC])
def test_branch_matrices_double_float(prec):
    """For K > 4 the FP32 paths form the branch matrices of reversible models
    in double-float arithmetic (float pairs, about 48 significant bits): every
    entry against the oracle's FP64 product (Eq. convolution) to 1e-11, for a
    61-state codon model over 3 epochs and a 20-state model."""
    cases = (synth.small_codon(204, n_taxa=10, n_sites=60, n_cat=2, n_epochs=3),
             synth.tiny_tree_workload(320, K=20, n_taxa=9, n_sites=50, n_epochs=3, n_cat=2))
    for w in cases:
        lik = EpochLikelihood(w, precision=prec)
        try:
            lik.log_likelihood()
            for v in range(2 * w.n_taxa - 2):
                for c in range(w.n_categories):
                    err = np.abs(lik.branch_matrix(v, c) - oracle.branch_matrix(w, v, c)).max()
                    assert err <= 1e-11, (w.K, v, c, err)
        finally:
            lik.close()


@pytest.mark.parametrize("prec", [EPOCH_FP64, EPOCH_FP32, EPOCH_FP32_TC])
def test_codon_small(prec):
    w = synth.small_codon(203, n_taxa=10, n_sites=120, n_cat=2, n_epochs=3)
    check_lnl(w, prec)
    check_grad(w, prec)


@pytest.mark.parametrize("prec", [EPOCH_FP64, EPOCH_FP32])
@pytest.mark.parametrize("K", [2, 3, 7, 20])
def test_other_state_counts(prec, K):
    w = synth.tiny_tree_workload(300 + K, K=K, n_taxa=9, n_sites=300, n_epochs=3, n_cat=2,
                                 missing_frac=0.05)
    check_lnl(w, prec)
    check_grad(w, prec)


@pytest.mark.parametrize("prec", [EPOCH_FP32_TC, EPOCH_FP32_TC_BF16])
@pytest.mark.parametrize("K,P", [(50, 300), (64, 129), (20, 257), (32, 130), (17, 140),
                                 (9, 200), (16, 131)])
def test_tensor_core_large_state_spaces(prec, K, P):
    """Tensor-core tiles: 64 wide for K = 50 asymmetric traits and K = 64 (no
    padding), 32 wide for K = 17, 20 and 32, 16 wide for K = 9 and 16; pattern
    counts that leave a ragged last tile of 128."""
    w = synth.tiny_tree_workload(320 + K, K=K, n_taxa=12, n_sites=P, n_epochs=3, n_cat=2,
                                 reversible=(K != 50), missing_frac=0.05)
    check_lnl(w, prec)
    check_grad(w, prec)


@pytest.mark.parametrize("prec", [EPOCH_FP64, EPOCH_FP32])
def test_asymmetric_uniformisation(prec):
    w = synth.tiny_tree_workload(310, K=12, n_taxa=8, n_sites=40, n_epochs=3, n_cat=1,
                                 reversible=False)
    check_lnl(w, prec)
    check_grad(w, prec)


@pytest.mark.parametrize("prec", [EPOCH_FP64, EPOCH_FP32])
def test_categories_and_single_epoch(prec):
    w = synth.small_nucleotide(204, n_taxa=30, n_sites=300, n_cat=8, n_epochs=1)
    check_lnl(w, prec)
    check_grad(w, prec)
    w1 = synth.small_nucleotide(205, n_taxa=30, n_sites=1, n_cat=1, n_epochs=2)
    check_lnl(w1, prec)


@pytest.mark.parametrize("prec", [EPOCH_FP64, EPOCH_FP32])
def test_shared_processes_phi(prec):
    """Alternating epochs sharing two processes (the paper's seasonal design)."""
    base = synth.small_nucleotide(206, n_taxa=30, n_sites=200, n_cat=2, n_epochs=5)
    phi = np.array([0, 1, 0, 1, 0], np.int32)
    w = base.replace(Q=base.Q[:2].copy(), epoch_to_matrix=phi,
                     dQ=np.ascontiguousarray(base.dQ[:12, :2]))
    check_lnl(w, prec)
    check_grad(w, prec)


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("prec", [EPOCH_FP64, EPOCH_FP32])
def test_zero_length_branch_and_node_on_boundary(prec):
    w = synth.small_nucleotide(207, n_taxa=12, n_sites=80, n_cat=2, n_epochs=3, dated=True)
    h = w.heights.copy()
    p = w.parent
    # a tip at the height of its parent (zero-length branch)
    t = 0
    h[t] = h[p[t]]
    # an internal node exactly on the first boundary
    u = next(v for v in range(w.n_taxa, 2 * w.n_taxa - 2)
             if h[p[v]] > w.boundaries[0] and max(h[c] for c in np.where(p == v)[0]) < w.boundaries[0])
    h[u] = w.boundaries[0]
    w2 = w.replace(heights=h)
    check_lnl(w2, prec)
    check_grad(w2, prec)


@pytest.mark.parametrize("prec", [EPOCH_FP64, EPOCH_FP32])
def test_missing_and_ambiguous_tips(prec):
    w = synth.small_nucleotide(208, n_taxa=15, n_sites=260, n_cat=2, n_epochs=2)
    rng = np.random.default_rng(0)
    tips = w.tips.copy()
    tips[rng.random(tips.shape) < 0.1] = 4                # missing
    masks = np.array([0b0101, 0b1010, 0b0011], np.uint64)  # purine, pyrimidine, AC
    sel = rng.random(tips.shape) < 0.1
    tips[sel] = 5 + rng.integers(0, 3, size=sel.sum())
    tips[3] = 4                                           # one tip entirely missing
    w2 = w.replace(tips=tips, masks=masks)
    check_lnl(w2, prec)
    check_grad(w2, prec)


@pytest.mark.parametrize("prec", [EPOCH_FP64, EPOCH_FP32])
def test_underflow_needs_scaling(prec):
    w = synth.small_nucleotide(209, n_taxa=600, n_sites=300, n_cat=2, n_epochs=3)
    rnd = np.random.default_rng(1).integers(0, 4, size=w.tips.shape).astype(np.int32)
    w = w.replace(tips=rnd, heights=w.heights * 40, boundaries=w.boundaries * 40)
    lnl = check_lnl(w, prec)
    assert lnl / w.pattern_weights.sum() < -709  # far below the FP64 range per site


# ---------------------------------------------------------------------------
# API behaviour on the device
# ---------------------------------------------------------------------------


def test_graph_replay_matches_direct_calls():
    w = synth.small_nucleotide(210, n_taxa=50, n_sites=600, n_cat=4, n_epochs=3)
    for prec in (EPOCH_FP64, EPOCH_FP32):
        lik = EpochLikelihood(w, precision=prec)
        try:
            lnl = lik.log_likelihood()
            g = lik.gradient()
            for _ in range(3):
                lnl2, g2 = lik.evaluate(with_gradient=True)
                assert lnl2 == lnl
                assert np.array_equal(g2["heights"], g["heights"])
                assert np.array_equal(g2["params"], g["params"])
            lnl3, _ = lik.evaluate(with_gradient=False)
            assert lnl3 == lnl
            # one graph each: partials only (log_likelihood), gradient only,
            # lnL + gradient, lnL
            launches, captures = lik.counters()
            assert launches > 0 and captures == 4
            # new heights, same topology: the captured graphs are reused
            h = w.heights * 1.1
            binding.epoch_set_heights(lik.ctx, h)
            lnl4, _ = lik.evaluate(with_gradient=True)
            assert lik.log_likelihood() == lnl4
            assert lik.counters()[1] == 4
            assert rel(lnl4, oracle.log_likelihood(w.replace(heights=h, boundaries=w.boundaries))[0]) \
                <= LNL_TOL[prec]
        finally:
            lik.close()


@pytest.mark.parametrize("n_cat,n_taxa,n_sites", [(1, 40, 333), (2, 3, 17), (3, 25, 130),
                                                    (5, 2, 9), (8, 60, 257)])
def test_repeated_and_interleaved_passes_k4(n_cat, n_taxa, n_sites):
    """The FP32 K = 4 pass keeps per-pattern exponent totals and a CTA
    counter on the device and leaves both zeroed for the next pass.  Repeated
    and interleaved calls (partials only, lnL + gradient, lnL only, new
    heights) must agree exactly with each other and with the oracle, for
    walks of 1, 2, 4 and 8 category lanes per pattern (C = 1, 2, 3, 5, 8),
    pattern counts that are not multiples of a walk CTA's patterns, and two-
    and three-taxon trees."""
    w = synth.small_nucleotide(230 + n_cat, n_taxa=n_taxa, n_sites=n_sites, n_cat=n_cat, n_epochs=3)
    lik = EpochLikelihood(w, precision=EPOCH_FP32)
    try:
        first = lik.log_likelihood()
        site = lik.site_log_likelihoods()
        for _ in range(3):
            assert lik.log_likelihood() == first
        lnl_g, g = lik.evaluate(with_gradient=True)
        lnl_n, _ = lik.evaluate(with_gradient=False)
        assert lnl_g == first and lnl_n == first
        assert np.array_equal(lik.site_log_likelihoods(), site)
        assert lik.log_likelihood() == first
        h = w.heights * 1.05
        binding.epoch_set_heights(lik.ctx, h)
        second = lik.log_likelihood()
        lnl2, _ = lik.evaluate(with_gradient=True)
        assert lnl2 == second
    finally:
        lik.close()
    rlnl, rsite = oracle.log_likelihood(w)
    assert rel(first, rlnl) <= LNL_TOL[EPOCH_FP32]
    assert np.allclose(site, rsite, rtol=1e-4, atol=1e-4 * np.abs(rsite).max())
    w2 = w.replace(heights=h, boundaries=w.boundaries)
    assert rel(second, oracle.log_likelihood(w2)[0]) <= LNL_TOL[EPOCH_FP32]


def test_errors_are_status_codes():
    w = synth.small_nucleotide(211, n_taxa=10, n_sites=20, n_cat=2, n_epochs=2)
    ctx = binding.epoch_create(4, 2, w.boundaries, None, 2, 10, 20, 2, EPOCH_FP32)
    try:
        with pytest.raises(EpochError) as e:
            binding.epoch_update_partials(ctx)
        assert e.value.status == 2  # out of order
        bad = w.Q.copy()
        bad[0, 0, 1] = -0.1
        with pytest.raises(EpochError) as e:
            binding.epoch_set_rate_matrices(ctx, bad, w.pi)
        assert e.value.status == 4
        asym = w.Q.copy()
        asym[0, 0, 1] += 0.3
        asym[0, 0, 0] -= 0.3
        with pytest.raises(EpochError) as e:
            binding.epoch_set_rate_matrices(ctx, asym, w.pi, 1, 1)
        assert e.value.status == 4  # claims reversibility it does not have
        with pytest.raises(EpochError) as e:
            binding.epoch_set_tree(ctx, *synth.coalescent_tree(11, np.random.default_rng(0)))
        assert e.value.status == 3  # more taxa than max_taxa
        binding.epoch_set_tree(ctx, w.heights, w.parent)
        tips = w.tips.copy()
        tips[0, 0] = 9
        with pytest.raises(EpochError) as e:
            binding.epoch_set_tip_data(ctx, tips, w.pattern_weights)
        assert e.value.status == 1
    finally:
        binding.epoch_destroy(ctx)


def test_impossible_pattern_gives_minus_infinity():
    """Two identical-height tips with different states on a zero-length
    cherry have probability 0: lnL = -inf is a result, not an error."""
    w = synth.small_nucleotide(212, n_taxa=6, n_sites=5, n_cat=1, n_epochs=2)
    h = w.heights.copy()
    p = w.parent
    u = next(x for x in range(w.n_taxa, 2 * w.n_taxa - 1)
             if (np.where(p == x)[0] < w.n_taxa).all())   # a cherry: both children tips
    kids = np.where(p == u)[0]
    h[kids] = h[u]
    tips = w.tips.copy()
    tips[kids[0], 0], tips[kids[1], 0] = 0, 1
    w2 = w.replace(heights=h, tips=tips)
    for prec in (EPOCH_FP64, EPOCH_FP32):
        lik = EpochLikelihood(w2, precision=prec)
        try:
            assert lik.log_likelihood() == -np.inf
            site = lik.site_log_likelihoods()
            impossible = tips[kids[0]] != tips[kids[1]]
            assert impossible[0]
            assert (site[impossible] == -np.inf).all() and np.isfinite(site[~impossible]).all()
        finally:
            lik.close()


@pytest.mark.parametrize("K,P", [(4, 300), (7, 200), (12, 150), (20, 257), (61, 130)])
def test_auto_path_is_the_faster_and_matches_the_oracle(K, P):
    """EPOCH_FP32_AUTO: the library times its SIMT and tensor-core FP32 paths
    on a synthetic problem of the same shape and keeps the faster (K <= 8:
    the SIMT path, no probe); a second context of the shape reuses the
    choice; the chosen path meets the FP32 tolerances against the oracle."""
    if K == 61:
        w = synth.small_codon(61, n_taxa=10, n_sites=P, n_cat=2, n_epochs=2).slice_patterns(0, P)
    else:
        w = synth.tiny_tree_workload(330 + K, K=K, n_taxa=14, n_sites=P, n_epochs=3, n_cat=2,
                                     missing_frac=0.05)
    lik = EpochLikelihood(w, precision=EPOCH_FP32_AUTO)
    try:
        info = binding.epoch_path_info(lik.ctx)
    finally:
        lik.close()
    prec, times = info[0], dict(zip((EPOCH_FP32, EPOCH_FP32_TC, EPOCH_FP32_TC_BF16), info[1:]))
    if K <= 8:
        assert prec == EPOCH_FP32 and all(t < 0 for t in times.values())
    else:
        assert all(t > 0 for t in times.values()), times
        assert prec == min(times, key=times.get), (prec, times)
    lik2 = EpochLikelihood(w, precision=EPOCH_FP32_AUTO)
    try:
        assert binding.epoch_path_info(lik2.ctx) == info
    finally:
        lik2.close()
    check_lnl(w, EPOCH_FP32_AUTO)
    check_grad(w, EPOCH_FP32_AUTO)


def test_one_call_step_equals_separate_calls():
    """epoch_evaluate_step sets the per-step inputs exactly as the setters and
    returns the results of epoch_evaluate_async + epoch_read_results; its
    errors are the setters' (a parent below its child: EPOCH_ERR_ARG)."""
    w = synth.small_nucleotide(808, n_taxa=20, n_sites=300, n_cat=4, n_epochs=3, dated=True)
    w2 = synth.small_nucleotide(809, n_taxa=20, n_sites=300, n_cat=4, n_epochs=3, dated=True)
    nn = 2 * w.n_taxa - 1
    for prec in (EPOCH_FP64, EPOCH_FP32):
        a = EpochLikelihood(w, precision=prec)
        b = EpochLikelihood(w, precision=prec)
        try:
            # new model and heights (w2's values on w's topology)
            h = np.array(w.heights) * 1.1
            Q, pi = np.ascontiguousarray(w2.Q, dtype=float), np.ascontiguousarray(w2.pi, dtype=float)
            dQ = np.ascontiguousarray(w.dQ, dtype=float)
            bd = np.ascontiguousarray(w.boundaries * 1.1)
            cr = np.ascontiguousarray(w.cat_rates, dtype=float)
            cw = np.ascontiguousarray(w.cat_weights, dtype=float)
            out = {"heights": np.zeros(nn), "boundaries": np.zeros(w.n_epochs - 1),
                   "params": np.zeros(a.n_params), "branch_rates": np.zeros(nn)}
            lnl = binding.epoch_evaluate_step(a.ctx, Q, pi, dQ, bd, cr, cw, h, True, out)
            binding.epoch_set_rate_matrices(b.ctx, Q, pi)
            binding.epoch_set_rate_derivatives(b.ctx, dQ)
            binding.epoch_set_boundaries(b.ctx, bd)
            binding.epoch_set_categories(b.ctx, cr, cw)
            binding.epoch_set_heights(b.ctx, h)
            binding.epoch_evaluate_async(b.ctx, True)
            lnl_b, g_b = binding.epoch_read_results(b.ctx, nn, w.n_epochs, b.n_params, True)
            assert lnl == lnl_b
            for k in ("heights", "boundaries", "params", "branch_rates"):
                assert np.array_equal(out[k], np.asarray(g_b[k])[: out[k].size]), k
            bad = h.copy()
            bad[int(np.where(np.asarray(w.parent) < 0)[0][0])] = -1.0
            with pytest.raises(EpochError) as e:
                binding.epoch_evaluate_step(a.ctx, Q, pi, heights=bad)
            assert e.value.status == 1
            # a refused step changed nothing
            assert binding.epoch_evaluate_step(a.ctx, out=out) == lnl

            # bound to fixed buffers, updated in place: only the heights are
            # given, the other inputs stay as the last step left them
            hbuf = h.copy()
            step = binding.epoch_step_function(a.ctx, heights=hbuf, out=out)
            hbuf *= 1.05
            lnl2 = step()
            binding.epoch_set_heights(b.ctx, h * 1.05)
            binding.epoch_evaluate_async(b.ctx, True)
            lnl2_b, g2_b = binding.epoch_read_results(b.ctx, nn, w.n_epochs, b.n_params, True)
            assert lnl2 == lnl2_b and lnl2 != lnl
            for k in ("heights", "boundaries", "params", "branch_rates"):
                assert np.array_equal(out[k], np.asarray(g2_b[k])[: out[k].size]), k

            # heights set from device memory survive a step that is given
            # other inputs (the host copy of the heights is stale then)
            import torch
            dh = torch.tensor(h * 0.95, dtype=torch.float64, device="cuda")
            binding.epoch_set_heights_device(a.ctx, dh.data_ptr())
            lnl3 = binding.epoch_evaluate_step(a.ctx, Q, pi, dQ, bd, cr, cw, None, False)
            binding.epoch_set_heights(b.ctx, h * 0.95)
            binding.epoch_evaluate_async(b.ctx, False)
            assert lnl3 == binding.epoch_read_results(b.ctx, nn, w.n_epochs, b.n_params, False)[0]
        finally:
            a.close()
            b.close()
