"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Nothing here compares the oracle with itself: each test checks it against a
closed form, an identity stated in the paper, a library routine on a special
case, brute-force enumeration, or finite differences.

  exp / a3       P(0) = I, rows sum to 1, P >= 0, detailed balance (Methods);
                 JC69 closed form; Jacobi eigensystem vs numpy; eigen path vs
                 uniformisation vs scipy.linalg.expm; Frechet derivative vs
                 scipy.linalg.expm_frechet.
  normalise      sum_i pi_i q_ii = -1 (Methods, after Eq. makeprobs).
  segments / a2  hand-built branches: inside one epoch, across every
                 boundary, ending on a boundary, zero length.
  product / a4   single epoch == homogeneous ("no new work", Relaxing
                 time-homogeneity); Chapman-Kolmogorov: a boundary between
                 identical Q changes nothing (Eq. matrixProduct); order: 2-state
                 closed forms with different (pi, mu) per epoch.
  pruning a5-a7  brute force over all internal states (K = 3, 4, 61);
                 two-taxon JC69 closed form; all-missing tip == tip removed;
                 duplicated site == weight 2; scaling on == off; permutation;
                 ambiguity masks: linearity in the tip indicator vector (a mask
                 tip's site likelihood is the sum over its states), full mask ==
                 missing, one-state mask == that state.
  gradient       central finite differences (h = 1e-6, FP64) for heights,
                 boundaries, branch rates and model parameters; d/db = 0
                 exactly when Q_k = Q_{k+1}; time-rescaling identity
                 sum h dh + sum b db = sum r dr.
"""
import numpy as np
import pytest
import scipy.linalg as sl

import synth

# ---------------------------------------------------------------------------
# helpers (test-side only)
# ---------------------------------------------------------------------------


def jc69_Q():
    Q = np.full((4, 4), 1.0 / 3.0)
    np.fill_diagonal(Q, -1.0)
    return Q


def two_state_P(pi1, mu, t):
    """Closed form of exp(t Q) for Q = mu [[-pi1, pi1], [pi0, -pi0]]."""
    pi0 = 1.0 - pi1
    e = np.exp(-mu * t)
    return np.array([[pi0 + pi1 * e, pi1 * (1 - e)], [pi0 * (1 - e), pi1 + pi0 * e]])


def two_state_Q(pi1, mu):
    pi0 = 1.0 - pi1
    return mu * np.array([[-pi1, pi1], [pi0, -pi0]])


def simple_workload(K, Q, pi, heights, parent, tips, boundaries=(), cat_rates=(1.0,),
                    cat_weights=(1.0,), normalise=1, reversible=1, weights=None,
                    phi=None, branch_rates=None, dQ=None):
    Q = np.asarray(Q, dtype=float)
    if Q.ndim == 2:
        Q = Q[None]
    E = len(boundaries) + 1
    tips = np.asarray(tips, dtype=np.int32)
    if tips.ndim == 1:
        tips = tips[:, None]
    if phi is None:
        phi = np.arange(E, dtype=np.int32) if Q.shape[0] == E else np.zeros(E, dtype=np.int32)
    return synth.Workload("t", K, np.asarray(boundaries, dtype=float), np.asarray(phi, np.int32), Q,
                          np.asarray(pi, float), np.asarray(cat_rates, float),
                          np.asarray(cat_weights, float), np.asarray(heights, float),
                          np.asarray(parent, np.int32), tips,
                          np.ones(tips.shape[1]) if weights is None else np.asarray(weights, float),
                          normalise=normalise, reversible=reversible, branch_rates=branch_rates,
                          dQ=dQ)


def rand_reversible(rng, K):
    pi = rng.dirichlet(np.full(K, 2.0))
    S = rng.lognormal(0, 0.8, size=(K, K))
    S = (S + S.T) / 2
    Q = S * pi[None, :]
    np.fill_diagonal(Q, 0)
    np.fill_diagonal(Q, -Q.sum(1))
    return Q, pi


def drop_tip(w, t):
    """Remove tip t and its parent; the sibling hangs from the grandparent.
    Relabels nodes so tips stay 0..N-2."""
    parent = w.parent.copy()
    p = parent[t]
    gp = parent[p]
    assert gp >= 0, "choose a tip whose parent is not the root"
    sib = [v for v in range(len(parent)) if parent[v] == p and v != t][0]
    parent[sib] = gp
    keep = [v for v in range(len(parent)) if v not in (t, p)]
    newid = {v: i for i, v in enumerate(keep)}
    N = w.n_taxa
    new_parent = np.array([newid[parent[v]] if parent[v] >= 0 else -1 for v in keep], np.int32)
    tips_keep = [v for v in keep if v < N]
    return w.replace(parent=new_parent, heights=w.heights[keep],
                     tips=np.ascontiguousarray(w.tips[tips_keep]))


# ---------------------------------------------------------------------------
# exp, eigen, normalisation (a1, a3)
# ---------------------------------------------------------------------------


def test_normalise_sets_expected_rate(oracle_lib):
    rng = np.random.default_rng(0)
    Q, pi = rand_reversible(rng, 5)
    Qn, c = oracle_lib.normalise(3.7 * Q, pi)
    assert np.isclose((pi * np.diag(Qn)).sum(), -1.0, rtol=0, atol=1e-15)
    assert np.allclose(Qn * c, 3.7 * Q, rtol=1e-15, atol=0)


def test_jc69_closed_form(oracle_lib):
    Q = jc69_Q()
    pi = np.full(4, 0.25)
    for t in [0.0, 1e-6, 0.05, 0.3, 1.7, 12.0]:
        same = 0.25 + 0.75 * np.exp(-4 * t / 3)
        diff = 0.25 - 0.25 * np.exp(-4 * t / 3)
        ref = np.full((4, 4), diff)
        np.fill_diagonal(ref, same)
        for rev in (True, False):
            P = oracle_lib.expm(Q, t, pi, reversible=rev)
            assert np.allclose(P, ref, rtol=0, atol=2e-15), (t, rev)


@pytest.mark.parametrize("K", [2, 4, 7, 20, 61])
def test_exp_properties_and_eigen(oracle_lib, K):
    rng = np.random.default_rng(K)
    Q, pi = rand_reversible(rng, K)
    Q, _ = oracle_lib.normalise(Q, pi)
    lam, V, Vi = oracle_lib.eig_sym(Q, pi)
    assert np.allclose(V @ Vi, np.eye(K), atol=1e-12)
    assert np.allclose(V @ np.diag(lam) @ Vi, Q, atol=1e-12)
    assert np.allclose(np.sort(lam), np.sort(np.linalg.eigvals(Q).real), atol=1e-11)
    assert np.allclose(oracle_lib.expm(Q, 0.0, pi), np.eye(K), atol=1e-14)
    for t in [0.01, 0.4, 3.0]:
        P = oracle_lib.expm(Q, t, pi, reversible=True)
        Pu = oracle_lib.expm(Q, t, pi, reversible=False)
        Ps = sl.expm(t * Q)
        assert np.allclose(P.sum(1), 1.0, atol=1e-13)
        assert (P > -1e-15).all()
        # detailed balance pi_i p_ij = pi_j p_ji
        D = pi[:, None] * P
        assert np.allclose(D, D.T, atol=1e-14)
        assert np.allclose(P, Ps, atol=1e-13, rtol=0)
        assert np.allclose(Pu, Ps, atol=1e-13, rtol=0)


def test_uniformisation_asymmetric_and_long_time(oracle_lib):
    rng = np.random.default_rng(5)
    K = 9
    R = rng.lognormal(0, 1, size=(K, K))
    np.fill_diagonal(R, 0)
    Q = R - np.diag(R.sum(1))
    for t in [0.0, 0.02, 1.0, 25.0]:   # 25 * max|q_ii| >> 30: repeated-multiplication path
        Pu = oracle_lib.expm(Q, t, reversible=False)
        assert np.allclose(Pu, sl.expm(t * Q), atol=1e-12, rtol=0)
        assert np.allclose(Pu.sum(1), 1.0, atol=1e-13)


def test_frechet_matches_scipy(oracle_lib):
    rng = np.random.default_rng(11)
    for K in (3, 8, 20):
        Q, pi = rand_reversible(rng, K)
        X = 0.7 * Q
        Y = rng.normal(size=(K, K))
        L = oracle_lib.frechet(X, Y)
        _, Lref = sl.expm_frechet(X, Y)
        assert np.allclose(L, Lref, rtol=1e-11, atol=1e-12)


# ---------------------------------------------------------------------------
# segmentation (a2)
# ---------------------------------------------------------------------------


def test_segments_hand_cases(oracle_lib):
    b = [1.0, 4.5]      # the shape of the paper's 5-taxon example (t1 = 1.0, t2 = 4.5)
    # inside epoch 0
    assert oracle_lib.segments(b, 0.2, 0.9, parent=7, child=3) == [(0, pytest.approx(0.7), 7, 3)]
    # crossing both boundaries, parent end first
    s = oracle_lib.segments(b, 0.5, 6.0, parent=8, child=2)
    assert [x[0] for x in s] == [2, 1, 0]
    assert np.allclose([x[1] for x in s], [1.5, 3.5, 0.5])
    assert [(x[2], x[3]) for x in s] == [(8, -2), (-2, -1), (-1, 2)]
    # child exactly on a boundary: the zero-length piece below it is dropped
    s = oracle_lib.segments(b, 1.0, 2.0, parent=5, child=1)
    assert s == [(1, pytest.approx(1.0), 5, 1)]
    # parent exactly on a boundary
    s = oracle_lib.segments(b, 2.0, 4.5, parent=5, child=1)
    assert s == [(1, pytest.approx(2.5), 5, 1)]
    # zero-length branch keeps one zero-length segment
    s = oracle_lib.segments(b, 3.0, 3.0, parent=5, child=1)
    assert s == [(1, 0.0, 5, 1)]
    # no boundaries at all
    assert oracle_lib.segments([], 0.0, 2.0, 1, 0) == [(0, pytest.approx(2.0), 1, 0)]
    # durations add up to the branch length
    rng = np.random.default_rng(1)
    bb = np.sort(rng.uniform(0, 10, 6))
    for _ in range(50):
        lo, hi = np.sort(rng.uniform(0, 12, 2))
        s = oracle_lib.segments(bb, lo, hi)
        assert np.isclose(sum(x[1] for x in s), hi - lo, rtol=0, atol=1e-12)
        eps = [x[0] for x in s]
        assert eps == sorted(eps, reverse=True)


# ---------------------------------------------------------------------------
# epoch products (a4)
# ---------------------------------------------------------------------------


def _cherry(H, h0=0.0, h1=0.0):
    return np.array([h0, h1, H]), np.array([2, 2, -1], np.int32)


def test_product_order_two_state_closed_form(oracle_lib):
    """Epoch 0 (young) and epoch 1 (old) carry 2-state processes with different
    (pi, mu).  The branch from the root (height H) to a tip at 0 crosses b:
    P = exp((H-b) Q_old) exp(b Q_young), the parent-end factor on the left
    (Eq. matrixProduct with rows = ancestral state)."""
    H, b = 1.3, 0.5
    Qy, Qo = two_state_Q(0.2, 1.5), two_state_Q(0.7, 0.4)
    heights, parent = _cherry(H)
    w = simple_workload(2, np.stack([Qy, Qo]), [0.5, 0.5], heights, parent, [0, 1],
                        boundaries=[b], normalise=0, reversible=0)
    ref = two_state_P(0.7, 0.4, H - b) @ two_state_P(0.2, 1.5, b)
    wrong = two_state_P(0.2, 1.5, b) @ two_state_P(0.7, 0.4, H - b)
    P = oracle_lib.branch_matrix(w, 0, 0)
    assert np.allclose(P, ref, atol=1e-14)
    assert not np.allclose(P, wrong, atol=1e-3)
    # swapping the epochs changes the result in the predicted way
    w2 = w.replace(Q=np.stack([Qo, Qy]))
    ref2 = two_state_P(0.2, 1.5, H - b) @ two_state_P(0.7, 0.4, b)
    assert np.allclose(oracle_lib.branch_matrix(w2, 0, 0), ref2, atol=1e-14)
    # two-taxon likelihood by hand: sum_i pi_i p_{i a} p_{i b}
    root_pi = np.array([0.5, 0.5])
    for a, c in [(0, 0), (0, 1), (1, 1)]:
        wt = w.replace(tips=np.array([[a], [c]], np.int32), pattern_weights=np.ones(1))
        L = sum(root_pi[i] * ref[i, a] * ref[i, c] for i in range(2))
        assert np.isclose(oracle_lib.log_likelihood(wt)[0], np.log(L), rtol=1e-14)


def test_single_epoch_equals_homogeneous(oracle_lib):
    rng = np.random.default_rng(3)
    Q, pi = rand_reversible(rng, 6)
    w = synth.tiny_tree_workload(7, K=6, n_taxa=6, n_sites=5, n_epochs=3)
    w_epoch = w.replace(Q=np.stack([Q, Q, Q]), pi=pi, dQ=None)
    w_homo = w.replace(Q=Q[None], pi=pi, boundaries=np.zeros(0),
                       epoch_to_matrix=np.zeros(1, np.int32), dQ=None)
    for v in range(2 * w.n_taxa - 2):
        for c in range(w.n_categories):
            Pe = oracle_lib.branch_matrix(w_epoch, v, c)
            Ph = oracle_lib.branch_matrix(w_homo, v, c)
            assert np.allclose(Pe, Ph, atol=1e-13)
            Qn, _ = oracle_lib.normalise(Q, pi)
            bl = w.heights[w.parent[v]] - w.heights[v]
            assert np.allclose(Ph, sl.expm(w.cat_rates[c] * bl * Qn), atol=1e-13)
    assert np.isclose(oracle_lib.log_likelihood(w_epoch)[0], oracle_lib.log_likelihood(w_homo)[0],
                      rtol=1e-13)


def test_chapman_kolmogorov_boundary_insertion(oracle_lib):
    """Adding or moving a boundary between identical processes leaves every
    branch matrix unchanged (Eq. matrixProduct)."""
    rng = np.random.default_rng(4)
    QA, pi = rand_reversible(rng, 4)
    QB, _ = rand_reversible(rng, 4)
    QB = QB * 0 + rand_reversible(np.random.default_rng(9), 4)[0]
    w = synth.tiny_tree_workload(8, K=4, n_taxa=7, n_sites=3, n_epochs=2)
    base = w.replace(Q=np.stack([QA, QB]), pi=pi, dQ=None)
    b1 = w.boundaries[0]
    # split epoch 1 into two with the same process, at a moved extra boundary
    for extra in (b1 + 0.11, b1 + 0.37):
        split = base.replace(boundaries=np.array([b1, extra]),
                             epoch_to_matrix=np.array([0, 1, 1], np.int32))
        for v in range(2 * w.n_taxa - 2):
            assert np.allclose(oracle_lib.branch_matrix(base, v, 0),
                               oracle_lib.branch_matrix(split, v, 0), atol=1e-13)
        assert np.isclose(oracle_lib.log_likelihood(base)[0], oracle_lib.log_likelihood(split)[0],
                          rtol=1e-13)


def test_branch_matrix_from_library_exponentials(oracle_lib):
    """Each branch = product of scipy exponentials of the (oracle-normalised,
    pinned above) Q over the (pinned above) segments, parent end first."""
    w = synth.tiny_tree_workload(12, K=5, n_taxa=6, n_sites=2, n_epochs=4, n_cat=3)
    Qn = np.stack([oracle_lib.normalise(q, w.pi)[0] for q in w.Q])
    for v in range(2 * w.n_taxa - 2):
        u = w.parent[v]
        segs = oracle_lib.segments(w.boundaries, w.heights[v], w.heights[u], u, v)
        for c in range(w.n_categories):
            M = np.eye(w.K)
            for (e, dt, _, _) in segs:
                M = M @ sl.expm(w.cat_rates[c] * dt * Qn[w.epoch_to_matrix[e]])
            assert np.allclose(oracle_lib.branch_matrix(w, v, c), M, atol=1e-13)


# ---------------------------------------------------------------------------
# pruning, root sum (a5-a7)
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("K,rev", [(3, True), (4, True), (4, False), (6, False)])
def test_pruning_equals_brute_force(oracle_lib, K, rev):
    for seed in range(3):
        w = synth.tiny_tree_workload(100 + seed, K=K, n_taxa=4, n_sites=5, n_epochs=3,
                                     n_cat=2, reversible=rev, missing_frac=0.15)
        lp, sp = oracle_lib.log_likelihood(w)
        lb, sb = oracle_lib.brute_force(w)
        assert np.isclose(lp, lb, rtol=1e-12)
        assert np.allclose(sp, sb, rtol=1e-12)


def test_pruning_equals_brute_force_codon(oracle_lib):
    w = synth.small_codon(21, n_taxa=4, n_sites=40, n_cat=1, n_epochs=2)
    w = w.slice_patterns(0, 2)
    lp, _ = oracle_lib.log_likelihood(w)
    lb, _ = oracle_lib.brute_force(w)
    assert np.isclose(lp, lb, rtol=1e-12)


def test_two_taxon_jc69_by_hand(oracle_lib):
    H, h1 = 0.8, 0.15
    heights, parent = _cherry(H, 0.0, h1)
    tips = np.array([[0, 0, 2, 3], [0, 1, 2, 1]], np.int32)
    w = simple_workload(4, jc69_Q(), np.full(4, 0.25), heights, parent, tips)

    def p(same, t):
        return 0.25 + 0.75 * np.exp(-4 * t / 3) if same else 0.25 - 0.25 * np.exp(-4 * t / 3)

    ref = []
    for a, c in tips.T:
        ref.append(np.log(sum(0.25 * p(i == a, H) * p(i == c, H - h1) for i in range(4))))
    _, site = oracle_lib.log_likelihood(w)
    assert np.allclose(site, ref, rtol=1e-14)


def test_missing_tip_equals_removed_tip(oracle_lib):
    w = synth.tiny_tree_workload(31, K=4, n_taxa=7, n_sites=6, n_epochs=3)
    root = int(np.where(w.parent < 0)[0][0])
    t = next(v for v in range(w.n_taxa) if w.parent[v] != root)
    tips = w.tips.copy()
    tips[t] = w.K
    wm = w.replace(tips=tips)
    wr = drop_tip(w, t)
    assert np.isclose(oracle_lib.log_likelihood(wm)[0], oracle_lib.log_likelihood(wr)[0],
                      rtol=1e-13)


def _with_tip_codes(w, changes):
    """Copy of w with tips[t, p] = code for every (t, p, code) in changes."""
    tips = w.tips.copy()
    for t, p, code in changes:
        tips[t, p] = code
    return w.replace(tips=tips)


@pytest.mark.parametrize("K,rev,cats", [(3, True, 1), (4, True, 2), (6, False, 2)])
def test_ambiguity_masks_are_sums_over_their_states(oracle_lib, K, rev, cats):
    """Pruning is linear in each tip's indicator vector (Eq. partial_likelihood:
    a tip's partial is 1 on every state it allows).  So a tip coded by the mask
    {i, j, ...} gives site likelihood L(tip = i) + L(tip = j) + ..., each term
    computed with the tip observed in one state.  Two mask tips in one pattern
    give the double sum.  Every pattern uses a different mask, so an off-by-one
    mask index or a reversed bit order changes the result."""
    rng = np.random.default_rng(7 + K)
    w = synth.tiny_tree_workload(60 + K, K=K, n_taxa=6, n_sites=8, n_epochs=3,
                                 n_cat=cats, reversible=rev)
    P = w.n_patterns
    full = (1 << K) - 1
    masks = []
    for _ in range(2 * P):
        while True:
            m = int(rng.integers(1, full))
            if bin(m).count("1") >= 2:
                break
        masks.append(m)
    masks = np.array(masks, np.uint64)
    t1, t2 = 1, 4
    w = w.replace(masks=masks)
    # one mask tip per pattern: tip t1 uses mask p
    wm = _with_tip_codes(w, [(t1, p, K + 1 + p) for p in range(P)])
    _, site_m = oracle_lib.log_likelihood(wm)
    per_state = np.array([oracle_lib.log_likelihood(
        _with_tip_codes(w, [(t1, p, s) for p in range(P)]))[1] for s in range(K)])
    for p in range(P):
        states = [s for s in range(K) if (int(masks[p]) >> s) & 1]
        ref = np.logaddexp.reduce(per_state[states, p])
        assert np.isclose(site_m[p], ref, rtol=1e-12, atol=1e-13), (p, site_m[p], ref)
    # two mask tips in the same pattern: t1 uses mask p, t2 uses mask P + p
    wm2 = _with_tip_codes(w, [(t, p, K + 1 + p + (P if t == t2 else 0))
                              for p in range(P) for t in (t1, t2)])
    _, site_m2 = oracle_lib.log_likelihood(wm2)
    pair = np.empty((K, K, P))
    for a in range(K):
        for b in range(K):
            pair[a, b] = oracle_lib.log_likelihood(
                _with_tip_codes(w, [(t, p, a if t == t1 else b)
                                    for p in range(P) for t in (t1, t2)]))[1]
    for p in range(P):
        sa = [s for s in range(K) if (int(masks[p]) >> s) & 1]
        sb = [s for s in range(K) if (int(masks[P + p]) >> s) & 1]
        ref = np.logaddexp.reduce([pair[a, b, p] for a in sa for b in sb])
        assert np.isclose(site_m2[p], ref, rtol=1e-12, atol=1e-13), (p, site_m2[p], ref)


def test_full_and_single_state_masks(oracle_lib):
    """A mask with every state set is the missing code K; a mask with one
    state set is that state's code (the tip's indicator vector is the same)."""
    K = 4
    w = synth.tiny_tree_workload(71, K=K, n_taxa=7, n_sites=6, n_epochs=2, n_cat=2)
    masks = np.array([(1 << K) - 1] + [1 << s for s in range(K)], np.uint64)
    w = w.replace(masks=masks)
    P = w.n_patterns
    for t in (0, 3, 6):
        full = _with_tip_codes(w, [(t, p, K + 1) for p in range(P)])
        miss = _with_tip_codes(w, [(t, p, K) for p in range(P)])
        assert np.allclose(oracle_lib.log_likelihood(full)[1],
                           oracle_lib.log_likelihood(miss)[1], rtol=1e-14)
        for s in range(K):
            one = _with_tip_codes(w, [(t, p, K + 2 + s) for p in range(P)])
            obs = _with_tip_codes(w, [(t, p, s) for p in range(P)])
            assert np.allclose(oracle_lib.log_likelihood(one)[1],
                               oracle_lib.log_likelihood(obs)[1], rtol=1e-14)


def test_mask_gradient_matches_central_differences(oracle_lib):
    """The adjoint reads tip indicator vectors too: with mask tips the height
    gradient still equals central differences of lnL (h = 1e-6, FP64)."""
    K = 4
    w = synth.tiny_tree_workload(73, K=K, n_taxa=6, n_sites=6, n_epochs=3, n_cat=2)
    masks = np.array([0b0101, 0b1010, 0b0111], np.uint64)
    P = w.n_patterns
    w = _with_tip_codes(w.replace(masks=masks),
                        [(p % w.n_taxa, p, K + 1 + p % 3) for p in range(P)])
    g = oracle_lib.gradient(w)
    N = w.n_taxa
    for u in range(N, 2 * N - 1):
        if w.parent[u] < 0:
            continue

        def f(x, u=u):
            h = w.heights.copy()
            h[u] = x
            return oracle_lib.log_likelihood(w.replace(heights=h))[0]

        _check(g["heights"][u], _fd(f, w.heights[u]), ("height", u))


def test_weights_duplication_permutation_scaling(oracle_lib):
    w = synth.small_nucleotide(41, n_taxa=12, n_sites=30, n_cat=3)
    l0, site = oracle_lib.log_likelihood(w)
    assert np.isclose(l0, (w.pattern_weights * site).sum(), rtol=1e-14)
    # duplicating a column == doubling its weight
    dup = w.replace(tips=np.concatenate([w.tips, w.tips[:, :1]], axis=1),
                    pattern_weights=np.concatenate([w.pattern_weights, w.pattern_weights[:1]]))
    dbl = w.replace(pattern_weights=w.pattern_weights * np.r_[2.0, np.ones(w.n_patterns - 1)])
    assert np.isclose(oracle_lib.log_likelihood(dup)[0], oracle_lib.log_likelihood(dbl)[0],
                      rtol=1e-14)
    # permutation of patterns
    perm = np.random.default_rng(0).permutation(w.n_patterns)
    wp = w.replace(tips=np.ascontiguousarray(w.tips[:, perm]), pattern_weights=w.pattern_weights[perm])
    assert np.isclose(oracle_lib.log_likelihood(wp)[0], l0, rtol=1e-13)
    # scaling on == off when nothing underflows
    assert np.isclose(oracle_lib.log_likelihood(w, scaling=False)[0], l0, rtol=1e-13)


def test_scaling_prevents_underflow(oracle_lib):
    """Site likelihoods far below the FP64 range (uniform random states on
    600 long branches) are finite with scaling and -inf without it."""
    w = synth.small_nucleotide(43, n_taxa=600, n_sites=4, n_cat=2)
    rnd = np.random.default_rng(0).integers(0, 4, size=w.tips.shape).astype(np.int32)
    w = w.replace(heights=w.heights * 60.0, boundaries=w.boundaries * 60.0, tips=rnd)
    l_on, site = oracle_lib.log_likelihood(w)
    assert np.isfinite(l_on)
    assert (site < -709).any()  # these site likelihoods are below FP64 range
    l_off, _ = oracle_lib.log_likelihood(w, scaling=False)
    assert not np.isfinite(l_off)


# ---------------------------------------------------------------------------
# gradient (a8-a10)
# ---------------------------------------------------------------------------


def _fd(f, x0, h=1e-6):
    return (f(x0 + h) - f(x0 - h)) / (2 * h)


def _check(g, fd, what):
    assert abs(g - fd) <= 2e-6 * max(1.0, abs(fd)), (what, g, fd)


@pytest.mark.parametrize("rev", [True, False])
def test_gradient_matches_central_differences(oracle_lib, rev):
    w = synth.tiny_tree_workload(51, K=4, n_taxa=6, n_sites=7, n_epochs=3, n_cat=2,
                                 reversible=rev, dated=True, missing_frac=0.1)
    w = w.replace(branch_rates=np.random.default_rng(2).uniform(0.6, 1.4, 2 * w.n_taxa - 1))
    g = oracle_lib.gradient(w)
    lnl = lambda ww: oracle_lib.log_likelihood(ww)[0]
    assert np.isclose(g["lnL"], lnl(w), rtol=1e-14)
    nn = 2 * w.n_taxa - 1
    for u in range(nn):
        def f(x, u=u):
            h = w.heights.copy()
            h[u] = x
            return lnl(w.replace(heights=h))
        _check(g["heights"][u], _fd(f, w.heights[u]), f"h{u}")
    for j in range(w.n_epochs - 1):
        def f(x, j=j):
            b = w.boundaries.copy()
            b[j] = x
            return lnl(w.replace(boundaries=b))
        _check(g["boundaries"][j], _fd(f, w.boundaries[j]), f"b{j}")
    for v in range(nn - 1):
        def f(x, v=v):
            r = w.branch_rates.copy()
            r[v] = x
            return lnl(w.replace(branch_rates=r))
        _check(g["branch_rates"][v], _fd(f, w.branch_rates[v]), f"r{v}")
    for a in range(w.n_params):
        f = lambda x, a=a: lnl(w.replace(Q=w.Q + x * w.dQ[a]))
        _check(g["params"][a], _fd(f, 0.0), f"theta{a}")


def test_gradient_codon_parameters(oracle_lib):
    w = synth.small_codon(61, n_taxa=5, n_sites=30, n_cat=2, n_epochs=2)
    g = oracle_lib.gradient(w)
    lnl = lambda ww: oracle_lib.log_likelihood(ww)[0]
    for a in range(w.n_params):
        f = lambda x, a=a: lnl(w.replace(Q=w.Q + x * w.dQ[a]))
        _check(g["params"][a], _fd(f, 0.0, h=1e-5), w.param_names[a])
    def fb(x):
        return lnl(w.replace(boundaries=np.array([x])))
    _check(g["boundaries"][0], _fd(fb, w.boundaries[0]), "b0")


def test_boundary_gradient_zero_for_identical_processes(oracle_lib):
    w = synth.tiny_tree_workload(52, K=4, n_taxa=8, n_sites=5, n_epochs=3)
    Q = w.Q.copy()
    Q[1] = Q[0]
    g = oracle_lib.gradient(w.replace(Q=Q, dQ=None))
    assert g["boundaries"][0] == 0.0
    assert g["boundaries"][1] != 0.0


def test_time_rescaling_identity(oracle_lib):
    """Scaling every time by alpha equals scaling every rate by alpha:
    sum_u h_u dlnL/dh_u + sum_k b_k dlnL/db_k = sum_v r_v dlnL/dr_v."""
    for seed, rev in [(53, True), (54, False)]:
        w = synth.tiny_tree_workload(seed, K=4, n_taxa=9, n_sites=6, n_epochs=4,
                                     reversible=rev, dated=True)
        w = w.replace(branch_rates=np.ones(2 * w.n_taxa - 1), dQ=None)
        g = oracle_lib.gradient(w)
        lhs = (w.heights * g["heights"]).sum() + (w.boundaries * g["boundaries"]).sum()
        rhs = (w.branch_rates * g["branch_rates"]).sum()
        assert np.isclose(lhs, rhs, rtol=1e-11, atol=1e-11)


def test_many_epochs_one_process_is_homogeneous(oracle_lib):
    """The seasonal shape with 13 epochs that all use one process: by
    Chapman-Kolmogorov the twelve boundaries change nothing (Eq.
    matrixProduct), so lnL equals the single-epoch lnL and every boundary
    derivative vanishes; with two alternating processes it differs."""
    w = synth.flu_seasonal(seed=21, n_taxa=40, n_processes=1, n_traits=5)
    one = w.replace(boundaries=np.zeros(0), epoch_to_matrix=np.zeros(1, np.int32))
    assert np.isclose(oracle_lib.log_likelihood(w)[0], oracle_lib.log_likelihood(one)[0],
                      rtol=1e-13)
    g = oracle_lib.gradient(w.replace(dQ=None))
    assert np.abs(g["boundaries"]).max() <= 1e-10 * np.abs(g["heights"]).max()
    w2 = synth.flu_seasonal(seed=21, n_taxa=40, n_processes=2, n_traits=5)
    g2 = oracle_lib.gradient(w2.replace(dQ=None))
    assert np.abs(g2["boundaries"]).max() > 1e-3


def test_expected_counts_are_rate_derivatives(oracle_lib):
    """Markov jump counts: with raw (unnormalised) matrices, the count of
    i -> j jumps in epoch e equals q_ij d lnL / d (Q_e)_ij with the diagonal
    held fixed (the jump factors of a path's density), checked by central
    differences of lnL; the per-branch and per-epoch sums agree and no
    count is negative."""
    w = synth.tiny_tree_workload(61, K=4, n_taxa=6, n_sites=7, n_epochs=3, n_cat=2,
                                 reversible=True, dated=True)
    w = w.replace(branch_rates=np.random.default_rng(5).uniform(0.7, 1.3, 2 * w.n_taxa - 1))
    per_branch, per_epoch = oracle_lib.expected_counts(w)
    assert np.allclose(per_branch.sum(0), per_epoch.sum(0), rtol=1e-12)
    assert per_branch.min() >= 0.0 and per_epoch.min() >= 0.0
    assert np.all(np.diagonal(per_branch, axis1=1, axis2=2) == 0.0)
    w0 = w.replace(normalise=0, reversible=0)
    _, pe0 = oracle_lib.expected_counts(w0)
    lnl = lambda ww: oracle_lib.log_likelihood(ww)[0]
    h = 1e-6
    for e in range(w.n_epochs):
        for i, j in [(0, 1), (1, 0), (2, 3), (3, 1)]:
            Qp, Qm = w0.Q.copy(), w0.Q.copy()
            Qp[e, i, j] += h
            Qm[e, i, j] -= h
            fd = (lnl(w0.replace(Q=Qp)) - lnl(w0.replace(Q=Qm))) / (2 * h)
            assert abs(w0.Q[e, i, j] * fd - pe0[e, i, j]) <= 1e-7 * max(1.0, pe0[e, i, j]), (e, i, j)
    # the counts do not depend on how Q is scaled: the normalised model with
    # the same effective rates gives the same counts
    pb_n, _ = oracle_lib.expected_counts(w.replace(normalise=1))
    Qn = np.stack([oracle_lib.normalise(w.Q[s], w.pi)[0] for s in range(w.n_matrices)])
    pb_raw, _ = oracle_lib.expected_counts(w.replace(Q=Qn, normalise=0))
    assert np.allclose(pb_n, pb_raw, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("K,rev,cats", [(4, True, 2), (3, False, 1), (5, True, 3)])
def test_ancestral_states_equal_enumeration(oracle_lib, K, rev, cats):
    """Marginal posterior of every internal node's state: the two-pass
    (outside x inside) computation against enumeration of every joint
    assignment of the internal states (missing data, several categories,
    an asymmetric model); rows sum to one."""
    w = synth.tiny_tree_workload(71 + K, K=K, n_taxa=5, n_sites=6, n_epochs=2, n_cat=cats,
                                 reversible=rev, dated=True, missing_frac=0.2)
    a = oracle_lib.ancestral_states(w)
    b = oracle_lib.ancestral_states(w, brute=True)
    assert a.shape == (w.n_taxa - 1, w.n_patterns, K)
    assert np.abs(a - b).max() <= 1e-13
    assert np.allclose(a.sum(-1), 1.0, atol=1e-13)
