"""Seeded synthetic workloads (trees, raw rate matrices, category rates, data).

No likelihood arithmetic lives here (see the package docstring).  Conventions
shared by both consumers:

* node ids: tips 0..N-1, internal nodes N..2N-2, ``parent[root] = -1``;
* heights: time before the youngest tip (the youngest tip has height 0);
* boundaries: heights b_1 < ... < b_{E-1}; epoch 0 = [0, b_1) is the youngest;
* ``Q[s]``: raw (un-normalised) rate matrix of process s, rows sum to 0;
  ``epoch_to_matrix[e]`` names the process active in epoch e;
* ``dQ[a][s]`` = d Q[s] / d theta_a of the raw matrices;
* tip codes: 0..K-1 observed state, K = missing (all states allowed).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
from scipy import special, stats

# ---------------------------------------------------------------------------
# containers
# ---------------------------------------------------------------------------


@dataclass
class Workload:
    name: str
    K: int
    boundaries: np.ndarray            # [E-1]
    epoch_to_matrix: np.ndarray       # [E] int32
    Q: np.ndarray                     # [S][K][K] raw
    pi: np.ndarray                    # [K]
    cat_rates: np.ndarray             # [C]
    cat_weights: np.ndarray           # [C]
    heights: np.ndarray               # [2N-1]
    parent: np.ndarray                # [2N-1] int32
    tips: np.ndarray                  # [N][P] int32
    pattern_weights: np.ndarray       # [P]
    normalise: int = 1
    reversible: int = 1
    branch_rates: Optional[np.ndarray] = None
    masks: Optional[np.ndarray] = None
    dQ: Optional[np.ndarray] = None   # [n_params][S][K][K]
    param_names: List[str] = field(default_factory=list)
    seed: int = 0

    @property
    def n_epochs(self) -> int:
        return int(len(self.boundaries)) + 1

    @property
    def n_matrices(self) -> int:
        return int(self.Q.shape[0])

    @property
    def n_taxa(self) -> int:
        return int(self.tips.shape[0])

    @property
    def n_patterns(self) -> int:
        return int(self.tips.shape[1])

    @property
    def n_categories(self) -> int:
        return int(len(self.cat_rates))

    @property
    def n_params(self) -> int:
        return 0 if self.dQ is None else int(self.dQ.shape[0])

    def replace(self, **kw) -> "Workload":
        d = dict(self.__dict__)
        d.update(kw)
        return Workload(**d)

    def slice_patterns(self, lo: int, hi: int) -> "Workload":
        return self.replace(tips=np.ascontiguousarray(self.tips[:, lo:hi]),
                            pattern_weights=np.ascontiguousarray(self.pattern_weights[lo:hi]))


@dataclass
class BatchWorkload:
    """Many independent trees of uneven size (the batched phylogeography case)."""
    name: str
    K: int
    trees: List[Workload]


# ---------------------------------------------------------------------------
# trees
# ---------------------------------------------------------------------------


def coalescent_tree(n: int, rng: np.random.Generator, root_height: float = 1.0,
                    tip_heights: Optional[np.ndarray] = None):
    """Kingman coalescent genealogy of n tips, rescaled so the root sits at
    ``root_height``.  With ``tip_heights`` (dated tips) lineages enter the
    process at their sampling heights.  Returns (heights[2n-1], parent[2n-1])."""
    if n < 2:
        raise ValueError("need at least two taxa")
    heights = np.zeros(2 * n - 1)
    parent = np.full(2 * n - 1, -1, dtype=np.int32)
    th = np.zeros(n) if tip_heights is None else np.asarray(tip_heights, dtype=np.float64)
    th = th - th.min()
    heights[:n] = th
    order = np.argsort(th, kind="stable")
    pending = [int(i) for i in order]
    active: List[int] = []
    t = 0.0
    nxt = n
    while pending or len(active) > 1:
        while pending and heights[pending[0]] <= t:
            active.append(pending.pop(0))
        k = len(active)
        if k < 2:
            t = heights[pending[0]]
            continue
        wait = rng.exponential(2.0 / (k * (k - 1)))
        if pending and t + wait > heights[pending[0]]:
            t = heights[pending[0]]
            continue
        t += wait
        a, b = rng.choice(k, size=2, replace=False)
        ca, cb = active[a], active[b]
        for idx in sorted((a, b), reverse=True):
            active.pop(idx)
        heights[nxt] = t
        parent[ca] = nxt
        parent[cb] = nxt
        active.append(nxt)
        nxt += 1
    root = 2 * n - 2
    heights = heights * (root_height / heights[root])
    heights[root] = root_height
    return heights, parent


# ---------------------------------------------------------------------------
# raw rate matrices (textbook definitions) and their parameter derivatives
# ---------------------------------------------------------------------------

NUC = "ACGT"  # state order for nucleotides


def _fill_diag(Q):
    Q = Q.copy()
    np.fill_diagonal(Q, 0.0)
    np.fill_diagonal(Q, -Q.sum(axis=1))
    return Q


def hky_raw(kappa: float, pi: np.ndarray):
    """HKY85: q_ij = pi_j * (kappa if i<->j is a transition).  Returns (Q, dQ/dkappa)."""
    pi = np.asarray(pi, dtype=np.float64)
    Q = np.zeros((4, 4))
    D = np.zeros((4, 4))
    for i in range(4):
        for j in range(4):
            if i == j:
                continue
            ts = {NUC[i], NUC[j]} in ({"A", "G"}, {"C", "T"})
            Q[i, j] = pi[j] * (kappa if ts else 1.0)
            D[i, j] = pi[j] if ts else 0.0
    return _fill_diag(Q), _fill_diag(D)


GTR_PAIRS = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]  # AC AG AT CG CT GT


def gtr_raw(s: np.ndarray, pi: np.ndarray):
    """GTR: q_ij = s_{ij} pi_j with symmetric exchangeabilities s (6 of them).
    Returns (Q, dQ[6]) with dQ[k] = dQ/ds_k."""
    pi = np.asarray(pi, dtype=np.float64)
    Q = np.zeros((4, 4))
    dQ = np.zeros((6, 4, 4))
    for k, (i, j) in enumerate(GTR_PAIRS):
        Q[i, j] = s[k] * pi[j]
        Q[j, i] = s[k] * pi[i]
        dQ[k, i, j] = pi[j]
        dQ[k, j, i] = pi[i]
    return _fill_diag(Q), np.stack([_fill_diag(d) for d in dQ])


# Standard genetic code (NCBI table 1), codons in TCAG order.
_BASES = "TCAG"
GENETIC_CODE = "FFLLSSSSYY**CC*WLLLLPPPPHHQQRRRRIIIMTTTTNNKKSSRRVVVVAAAADDEEGGGG"
SENSE_CODONS = [i for i in range(64) if GENETIC_CODE[i] != "*"]


def _codon_nts(idx):
    return (idx // 16, (idx // 4) % 4, idx % 4)


def gy94_raw(kappa: float, omega: float, pi: np.ndarray):
    """Goldman-Yang 1994 on the 61 sense codons: codons differing at one
    position exchange at pi_j * (kappa if transition) * (omega if
    non-synonymous); all other off-diagonal rates are zero.
    Returns (Q, dQ/dkappa, dQ/domega)."""
    pi = np.asarray(pi, dtype=np.float64)
    n = len(SENSE_CODONS)
    Q = np.zeros((n, n))
    Dk = np.zeros((n, n))
    Dw = np.zeros((n, n))
    for a, ci in enumerate(SENSE_CODONS):
        xi = _codon_nts(ci)
        for b, cj in enumerate(SENSE_CODONS):
            if a == b:
                continue
            xj = _codon_nts(cj)
            diff = [p for p in range(3) if xi[p] != xj[p]]
            if len(diff) != 1:
                continue
            p = diff[0]
            pair = {_BASES[xi[p]], _BASES[xj[p]]}
            ts = pair in ({"T", "C"}, {"A", "G"})
            syn = GENETIC_CODE[ci] == GENETIC_CODE[cj]
            k = kappa if ts else 1.0
            w = 1.0 if syn else omega
            Q[a, b] = pi[b] * k * w
            Dk[a, b] = pi[b] * w if ts else 0.0
            Dw[a, b] = 0.0 if syn else pi[b] * k
    return _fill_diag(Q), _fill_diag(Dk), _fill_diag(Dw)


def codon_frequencies_f3x4(rng: np.random.Generator, conc: float = 10.0):
    """F3x4: codon frequency = product of three position-specific nucleotide
    frequencies (each ~ Dirichlet(conc*1)), renormalised over sense codons."""
    f = [rng.dirichlet(np.full(4, conc)) for _ in range(3)]
    pi = np.array([f[0][_codon_nts(c)[0]] * f[1][_codon_nts(c)[1]] * f[2][_codon_nts(c)[2]]
                   for c in SENSE_CODONS])
    return pi / pi.sum()


def asym_raw(rates: np.ndarray):
    """Asymmetric discrete-trait CTMC: q_ij = rates_ij for i != j."""
    return _fill_diag(np.asarray(rates, dtype=np.float64))


# ---------------------------------------------------------------------------
# among-site rate categories
# ---------------------------------------------------------------------------


def discrete_gamma(alpha: float, C: int):
    """Yang (1994) discrete gamma, mean-of-category rates with equal weights:
    r_c = C * [I(alpha+1, alpha*q_{c+1}) - I(alpha+1, alpha*q_c)] where q_c are
    the c/C quantiles of Gamma(alpha, rate alpha) and I the regularised lower
    incomplete gamma.  Mean rate is exactly 1."""
    if C == 1:
        return np.ones(1), np.ones(1)
    q = stats.gamma.ppf(np.arange(1, C) / C, a=alpha, scale=1.0 / alpha)
    edges = np.concatenate([[0.0], q, [np.inf]])
    cdf1 = special.gammainc(alpha + 1.0, alpha * edges)
    cdf1[-1] = 1.0
    rates = C * np.diff(cdf1)
    return rates, np.full(C, 1.0 / C)


# ---------------------------------------------------------------------------
# jump-chain simulation along an epoch tree
# ---------------------------------------------------------------------------


def _sim_rate_matrices(Qraw, pi, normalise):
    """Per-process rate matrices the simulator runs: the raw Q divided by its
    expected rate sum_i pi_i |q_ii| when the likelihood normalises."""
    out = []
    for Q in Qraw:
        if normalise:
            out.append(Q / float(-(pi * np.diag(Q)).sum()))
        else:
            out.append(Q.copy())
    return out


def simulate_alignment(heights, parent, boundaries, epoch_to_matrix, Qraw, pi, cat_rates,
                       n_sites, rng, normalise=True, branch_rates=None, root_pi=None):
    """Simulate n_sites columns by exact CTMC path simulation (Gillespie).
    Each site draws a category uniformly; along a branch the process runs
    from the parent's height down to the child's, switching to the epoch's
    Q at every boundary crossed.  Returns tip states [N][n_sites] int32."""
    nn = len(parent)
    N = (nn + 1) // 2
    K = Qraw[0].shape[0]
    b = np.asarray(boundaries, dtype=np.float64).reshape(-1)
    Qs = _sim_rate_matrices(Qraw, np.asarray(pi), normalise)
    phi = np.asarray(epoch_to_matrix, dtype=np.int64)
    # jump distributions per process
    exit_rate = np.stack([-np.diag(Q) for Q in Qs])                  # [S][K]
    jump = []
    for Q in Qs:
        R = Q.copy()
        np.fill_diagonal(R, 0.0)
        tot = R.sum(axis=1, keepdims=True)
        tot[tot == 0] = 1.0
        jump.append(np.cumsum(R / tot, axis=1))
    jump = np.stack(jump)                                             # [S][K][K]
    cats = rng.integers(0, len(cat_rates), size=n_sites)
    site_rate = np.asarray(cat_rates)[cats]
    state = np.zeros((nn, n_sites), dtype=np.int64)
    root = int(np.where(parent < 0)[0][0])
    rp = np.asarray(root_pi if root_pi is not None else pi, dtype=np.float64)
    state[root] = rng.choice(K, size=n_sites, p=rp / rp.sum())
    # breadth-first levels from the root
    children = [[] for _ in range(nn)]
    for v in range(nn):
        if parent[v] >= 0:
            children[parent[v]].append(v)
    level = [root]
    while level:
        nxt = [c for u in level for c in children[u]]
        if not nxt:
            break
        vs = np.array(nxt)
        us = parent[vs]
        nb = len(vs)
        st = state[us].copy()
        h = np.repeat(heights[us][:, None], n_sites, axis=1)
        hend = np.repeat(heights[vs][:, None], n_sites, axis=1)
        br = np.ones(nb) if branch_rates is None else np.asarray(branch_rates)[vs]
        mult = br[:, None] * site_rate[None, :]
        st = st.reshape(-1)
        h = h.reshape(-1)
        hend = hend.reshape(-1)
        mult = mult.reshape(-1)
        active = h > hend
        while active.any():
            idx = np.nonzero(active)[0]
            hh = h[idx]
            # epoch of the interval just below the current height
            e = np.searchsorted(b, hh, side="left")
            low = np.concatenate([[-np.inf], b])[e]
            seg_end = np.maximum(hend[idx], low)
            s = phi[e]
            lam = exit_rate[s, st[idx]] * mult[idx]
            with np.errstate(divide="ignore"):
                wait = np.where(lam > 0, rng.exponential(1.0, size=idx.size) / np.where(lam > 0, lam, 1.0), np.inf)
            jumps = hh - wait > seg_end
            # advance to the segment end where no jump happens
            h[idx[~jumps]] = seg_end[~jumps]
            if jumps.any():
                j_idx = idx[jumps]
                h[j_idx] = hh[jumps] - wait[jumps]
                u = rng.random(j_idx.size)
                cum = jump[s[jumps], st[j_idx]]                      # [n][K]
                st[j_idx] = np.minimum((u[:, None] >= cum).sum(axis=1), K - 1)
            active = h > hend
        state[vs] = st.reshape(nb, n_sites)
        level = nxt
    return np.ascontiguousarray(state[:N].astype(np.int32))


def compress_patterns(aln: np.ndarray):
    """Unique site columns and their multiplicities."""
    cols, counts = np.unique(aln.T, axis=0, return_counts=True)
    return np.ascontiguousarray(cols.T.astype(np.int32)), counts.astype(np.float64)


# ---------------------------------------------------------------------------
# workloads shaped like the paper's nucleotide, codon and trait analyses (seeds 1310-1314)
# ---------------------------------------------------------------------------


def _epoch_bounds(root, fracs):
    return np.array([root * f for f in fracs], dtype=np.float64)


def hky_8taxa(seed: int = 1310, n_taxa: int = 8, n_sites: int = 200) -> Workload:
    """Plain FP64 epoch likelihood: 8-taxon coalescent (root 1.0), HKY with
    kappa_e ~ LogN(1, 0.5) per epoch, pi ~ Dirichlet(1), 2 epochs split at 0.5,
    200 simulated sites compressed to unique patterns, one rate category."""
    rng = np.random.default_rng(seed)
    heights, parent = coalescent_tree(n_taxa, rng)
    pi = rng.dirichlet(np.ones(4))
    kap = rng.lognormal(1.0, 0.5, size=2)
    Qs, dQs = zip(*[hky_raw(k, pi) for k in kap])
    Q = np.stack(Qs)
    dQ = np.zeros((2, 2, 4, 4))
    dQ[0, 0] = dQs[0]
    dQ[1, 1] = dQs[1]
    b = _epoch_bounds(1.0, [0.5])
    phi = np.arange(2, dtype=np.int32)
    aln = simulate_alignment(heights, parent, b, phi, Q, pi, np.ones(1), n_sites, rng)
    tips, w = compress_patterns(aln)
    return Workload("hky-2epoch-8taxa", 4, b, phi, Q, pi, np.ones(1), np.ones(1), heights,
                    parent, tips, w, dQ=dQ, param_names=["kappa_0", "kappa_1"], seed=seed)


def _gtr_workload(name, seed, n_taxa, n_sites, n_cat, alpha, fracs, dated=False,
                  weights_uniform=(1, 20)):
    rng = np.random.default_rng(seed)
    th = rng.uniform(0.0, 0.2, size=n_taxa) if dated else None
    heights, parent = coalescent_tree(n_taxa, rng, tip_heights=th)
    E = len(fracs) + 1
    pi = rng.dirichlet(np.ones(4))
    Qs, dQs = [], []
    for _ in range(E):
        s = rng.lognormal(0.0, 1.0, size=6)
        Qe, dQe = gtr_raw(s, pi)
        Qs.append(Qe)
        dQs.append(dQe)
    Q = np.stack(Qs)
    dQ = np.zeros((6 * E, E, 4, 4))
    names = []
    for e in range(E):
        for k in range(6):
            dQ[6 * e + k, e] = dQs[e][k]
            names.append(f"s{''.join(NUC[x] for x in GTR_PAIRS[k])}_{e}")
    b = _epoch_bounds(1.0, fracs)
    phi = np.arange(E, dtype=np.int32)
    rates, cw = discrete_gamma(alpha, n_cat)
    aln = simulate_alignment(heights, parent, b, phi, Q, pi, rates, n_sites, rng)
    # one column per pattern, integer weights
    w = rng.integers(weights_uniform[0], weights_uniform[1] + 1, size=n_sites).astype(np.float64)
    return Workload(name, 4, b, phi, Q, pi, rates, cw, heights, parent, aln, w, dQ=dQ,
                    param_names=names, seed=seed)


def gtr_500taxa(seed: int = 1311, n_taxa: int = 500, n_sites: int = 10_000, dated=False) -> Workload:
    """GTR (exchangeabilities ~ LogN(0,1) per epoch, pi ~ Dirichlet(1)), 3 epochs
    at 1/3 and 2/3 of the root height, 500-taxon coalescent, 10,000 simulated
    columns each its own pattern with weight ~ U{1..20}, 4 discrete-gamma
    categories (alpha = 0.5)."""
    return _gtr_workload(f"gtr-3epoch-{n_taxa}taxa-{n_sites}p", seed, n_taxa, n_sites, 4, 0.5,
                         [1 / 3, 2 / 3], dated=dated)


def small_nucleotide(seed: int, n_taxa: int, n_sites: int, n_cat: int = 4, n_epochs: int = 3,
                     dated: bool = False) -> Workload:
    fracs = [k / n_epochs for k in range(1, n_epochs)]
    return _gtr_workload(f"gtr-{n_epochs}epoch-{n_taxa}taxa-{n_sites}p", seed, n_taxa, n_sites,
                         n_cat, 0.5, fracs, dated=dated)


def _gy94_workload(name, seed, n_taxa, n_sites, n_cat, fracs, kappa=2.0, dated=False,
                   compress=True):
    rng = np.random.default_rng(seed)
    th = rng.uniform(0.0, 0.2, size=n_taxa) if dated else None
    heights, parent = coalescent_tree(n_taxa, rng, tip_heights=th)
    E = len(fracs) + 1
    pi = codon_frequencies_f3x4(rng)
    omegas = rng.lognormal(-1.0, 0.7, size=E)
    Qs, Dk, Dw = [], [], []
    for e in range(E):
        q, dk, dw = gy94_raw(kappa, omegas[e], pi)
        Qs.append(q)
        Dk.append(dk)
        Dw.append(dw)
    Q = np.stack(Qs)
    K = Q.shape[1]
    dQ = np.zeros((1 + E, E, K, K))
    for e in range(E):
        dQ[0, e] = Dk[e]
        dQ[1 + e, e] = Dw[e]
    names = ["kappa"] + [f"omega_{e}" for e in range(E)]
    b = _epoch_bounds(1.0, fracs)
    phi = np.arange(E, dtype=np.int32)
    rates, cw = discrete_gamma(0.5, n_cat)
    aln = simulate_alignment(heights, parent, b, phi, Q, pi, rates, n_sites, rng)
    if compress:
        tips, w = compress_patterns(aln)
    else:
        tips, w = aln, np.ones(n_sites)
    return Workload(name, K, b, phi, Q, pi, rates, cw, heights, parent, tips, w, dQ=dQ,
                    param_names=names, seed=seed)


def gy94_128taxa(seed: int = 1312, n_taxa: int = 128, n_sites: int = 5000, dated=False) -> Workload:
    """GY94 (61 sense codons), kappa = 2 shared, omega_k ~ LogN(-1, 0.7) for 4
    epochs with boundaries at 1/4, 1/2, 3/4 of the root height, 128-taxon
    coalescent, 5,000 simulated codon sites compressed to patterns, 4
    discrete-gamma categories (alpha = 0.5), pi = F3x4."""
    return _gy94_workload(f"gy94-4epoch-{n_taxa}taxa-{n_sites}sites", seed, n_taxa, n_sites, 4,
                          [0.25, 0.5, 0.75], dated=dated)


def small_codon(seed: int, n_taxa: int, n_sites: int, n_cat: int = 2, n_epochs: int = 2,
                dated: bool = False) -> Workload:
    fracs = [k / n_epochs for k in range(1, n_epochs)]
    return _gy94_workload(f"gy94-{n_epochs}epoch-{n_taxa}taxa-{n_sites}s", seed, n_taxa, n_sites,
                          n_cat, fracs, dated=dated)


def _asym_tree(rng, K, n_taxa, n_epochs, n_pat, name):
    heights, parent = coalescent_tree(n_taxa, rng)
    b = np.sort(rng.uniform(0.0, 1.0, size=n_epochs - 1)) * heights[-1]
    Q = np.stack([asym_raw(rng.lognormal(0.0, 1.0, size=(K, K))) for _ in range(n_epochs)])
    pi = np.full(K, 1.0 / K)
    phi = np.arange(n_epochs, dtype=np.int32)
    aln = simulate_alignment(heights, parent, b, phi, Q, pi, np.ones(1), n_pat, rng)
    return Workload(name, K, b, phi, Q, pi, np.ones(1), np.ones(1), heights, parent, aln,
                    np.ones(n_pat), reversible=0)


def asym50_forest(seed: int = 1314, n_trees: int = 256, K: int = 50, taxa=(50, 1000), epochs=(1, 8),
            patterns=(1, 4)) -> BatchWorkload:
    """Batched phylogeography: n_trees independent coalescent trees (root 1.0)
    with N_t ~ U{50..1000} taxa, E_t ~ U{1..8} epochs at sorted U(0,1) heights,
    a K=50 asymmetric CTMC per epoch (off-diagonal rates ~ LogN(0,1)), pi
    uniform, P_t ~ U{1..4} simulated trait patterns, one rate category."""
    rng = np.random.default_rng(seed)
    trees = []
    for t in range(n_trees):
        n = int(rng.integers(taxa[0], taxa[1] + 1))
        E = int(rng.integers(epochs[0], epochs[1] + 1))
        P = int(rng.integers(patterns[0], patterns[1] + 1))
        trees.append(_asym_tree(rng, K, n, E, P, f"tree{t}"))
    return BatchWorkload(f"asym{K}-{n_trees}trees", K, trees)


def tiny_tree_workload(seed: int, K: int = 4, n_taxa: int = 4, n_sites: int = 6, n_epochs: int = 2,
                       n_cat: int = 2, reversible: bool = True, dated: bool = True,
                       missing_frac: float = 0.0) -> Workload:
    """Small random problems for brute-force and edge-case tests (any K)."""
    rng = np.random.default_rng(seed)
    th = rng.uniform(0.0, 0.3, size=n_taxa) if dated else None
    heights, parent = coalescent_tree(n_taxa, rng, tip_heights=th)
    b = np.sort(rng.uniform(0.05, 0.95, size=n_epochs - 1)) * heights[-1]
    if reversible:
        pi = rng.dirichlet(np.full(K, 3.0))
        Qs, dQs = [], []
        for _ in range(n_epochs):
            S = rng.lognormal(0.0, 0.7, size=(K, K))
            S = (S + S.T) / 2
            q = S * pi[None, :]
            Qs.append(_fill_diag(q))
            # one parameter per epoch: a global multiplier on the transition
            # between states 0 and 1 (exchangeability s_01)
            d = np.zeros((K, K))
            d[0, 1] = pi[1]
            d[1, 0] = pi[0]
            dQs.append(_fill_diag(d))
        Q = np.stack(Qs)
        dQ = np.zeros((n_epochs, n_epochs, K, K))
        for e in range(n_epochs):
            dQ[e, e] = dQs[e] * 1.0
        names = [f"s01_{e}" for e in range(n_epochs)]
    else:
        pi = np.full(K, 1.0 / K)
        Q = np.stack([asym_raw(rng.lognormal(0.0, 1.0, size=(K, K))) for _ in range(n_epochs)])
        dQ = None
        names = []
    phi = np.arange(n_epochs, dtype=np.int32)
    rates, cw = discrete_gamma(0.7, n_cat) if n_cat > 1 else (np.ones(1), np.ones(1))
    aln = simulate_alignment(heights, parent, b, phi, Q, pi, rates, n_sites, rng)
    if missing_frac > 0:
        miss = rng.random(aln.shape) < missing_frac
        aln = np.where(miss, K, aln).astype(np.int32)
    w = rng.integers(1, 4, size=n_sites).astype(np.float64)
    return Workload(f"tiny-K{K}-{n_taxa}taxa", K, b, phi, Q, pi, rates, cw, heights, parent,
                    aln, w, reversible=int(reversible), dQ=dQ, param_names=names, seed=seed)


def exchange_raw(s: np.ndarray, pi: np.ndarray):
    """General time-reversible K-state CTMC from K(K-1)/2 exchangeabilities
    (pairs (i, j), i < j, in row order): q_ij = s_ij pi_j.  Returns (Q, dQ)
    with dQ[k] = dQ/ds_k."""
    pi = np.asarray(pi, dtype=np.float64)
    K = len(pi)
    pairs = [(i, j) for i in range(K) for j in range(i + 1, K)]
    Q = np.zeros((K, K))
    dQ = np.zeros((len(pairs), K, K))
    for k, (i, j) in enumerate(pairs):
        Q[i, j] = s[k] * pi[j]
        Q[j, i] = s[k] * pi[i]
        dQ[k, i, j] = pi[j]
        dQ[k, j, i] = pi[i]
    return _fill_diag(Q), np.stack([_fill_diag(d) for d in dQ])


def flu_seasonal(seed: int = 1315, n_taxa: int = 522, K: int = 7, n_epochs: int = 13,
                 n_processes: int = 2, n_traits: int = 1, reversible: bool = True,
                 sampling_span: float = 0.4) -> Workload:
    """Seasonal phylogeography shaped like the paper's influenza analysis
    (Results, seasonal H3N2): n_taxa dated tips (heights ~ U(0, span) of a
    coalescent tree rescaled to root 1.0), K discrete locations, n_epochs
    epochs of equal length (boundaries k / n_epochs of the root height) that
    alternate between n_processes rate matrices (phi_e = e mod n_processes,
    the seasonal design), one simulated location trait per taxon (n_traits
    replicate traits, each its own pattern, weight 1), one rate category.

    reversible: exchange rates s_ij ~ LogN(0, 1) per process with pi uniform
    (the symmetric location-exchange model; the parameters are the K(K-1)/2
    exchangeabilities of each process); else asymmetric q_ij ~ LogN(0, 1),
    pi uniform, no model parameters."""
    rng = np.random.default_rng(seed)
    th = rng.uniform(0.0, sampling_span, size=n_taxa)
    heights, parent = coalescent_tree(n_taxa, rng, tip_heights=th)
    pi = np.full(K, 1.0 / K)
    npair = K * (K - 1) // 2
    if reversible:
        Qs, dQs = zip(*[exchange_raw(rng.lognormal(0.0, 1.0, size=npair), pi)
                        for _ in range(n_processes)])
        Q = np.stack(Qs)
        dQ = np.zeros((npair * n_processes, n_processes, K, K))
        names = []
        for s in range(n_processes):
            dQ[npair * s:npair * (s + 1), s] = dQs[s]
            names += [f"s{i}{j}_{s}" for i in range(K) for j in range(i + 1, K)]
    else:
        Q = np.stack([asym_raw(rng.lognormal(0.0, 1.0, size=(K, K))) for _ in range(n_processes)])
        dQ, names = None, []
    b = np.arange(1, n_epochs, dtype=np.float64) / n_epochs
    phi = (np.arange(n_epochs) % n_processes).astype(np.int32)
    aln = simulate_alignment(heights, parent, b, phi, Q, pi, np.ones(1), n_traits, rng)
    return Workload(f"seasonal-K{K}-{n_epochs}epoch-{n_taxa}taxa", K, b, phi, Q, pi, np.ones(1),
                    np.ones(1), heights, parent, aln, np.ones(n_traits), reversible=int(reversible),
                    dQ=dQ, param_names=names, seed=seed)


def amino_acid(seed: int = 1316, n_taxa: int = 200, n_sites: int = 2000, n_epochs: int = 3,
               n_cat: int = 4, K: int = 20, dated: bool = False) -> Workload:
    """Protein-shaped data: K = 20 states, a general time-reversible matrix
    per epoch (190 exchangeabilities ~ LogN(0, 1), pi ~ Dirichlet(10 * 1)
    shared), epochs at equal fractions of the root height, coalescent tree
    with root 1.0, simulated sites compressed to patterns, discrete-gamma
    categories (alpha = 0.5).  Parameters: the first three exchangeabilities
    (pairs 01, 02, 03) of each epoch."""
    rng = np.random.default_rng(seed)
    th = rng.uniform(0.0, 0.2, size=n_taxa) if dated else None
    heights, parent = coalescent_tree(n_taxa, rng, tip_heights=th)
    pi = rng.dirichlet(np.full(K, 10.0))
    npair = K * (K - 1) // 2
    Qs, dQs = zip(*[exchange_raw(rng.lognormal(0.0, 1.0, size=npair), pi) for _ in range(n_epochs)])
    Q = np.stack(Qs)
    dQ = np.zeros((3 * n_epochs, n_epochs, K, K))
    names = []
    for e in range(n_epochs):
        dQ[3 * e:3 * e + 3, e] = dQs[e][:3]
        names += [f"s01_{e}", f"s02_{e}", f"s03_{e}"]
    b = _epoch_bounds(1.0, [k / n_epochs for k in range(1, n_epochs)])
    phi = np.arange(n_epochs, dtype=np.int32)
    rates, cw = discrete_gamma(0.5, n_cat) if n_cat > 1 else (np.ones(1), np.ones(1))
    aln = simulate_alignment(heights, parent, b, phi, Q, pi, rates, n_sites, rng)
    tips, w = compress_patterns(aln)
    return Workload(f"aa-K{K}-{n_epochs}epoch-{n_taxa}taxa-{n_sites}s", K, b, phi, Q, pi, rates, cw,
                    heights, parent, tips, w, dQ=dQ, param_names=names, seed=seed)
