"""FP64 CPU oracle for the epoch-model tree likelihood (arXiv 1309.3075).

TEST INFRASTRUCTURE ONLY.  This package may be imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py``.
The product library (``paper_1309_3075_b300``) never imports it, and the two
share no code: the oracle is plain C (``epoch_oracle.c``) written from the
paper's definitions (Methods, Eq. makeprobs, Eq. partial_likelihood,
Eq. matrixProduct, Eq. convolution); this module only marshals numpy arrays.

Every function here is pinned in ``tests/test_oracle_pins.py`` against closed
forms, identities and brute force (see the module docstring there).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "epoch_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "epoch_oracle.h"))
    ):
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-o", _LIB_PATH, _SRC, "-lm"]
        subprocess.run(cmd, check=True, cwd=_HERE)
    return _LIB_PATH


class _Problem(C.Structure):
    _fields_ = [
        ("K", C.c_int),
        ("n_epochs", C.c_int),
        ("boundaries", C.POINTER(C.c_double)),
        ("epoch_to_matrix", C.POINTER(C.c_int)),
        ("n_matrices", C.c_int),
        ("Q", C.POINTER(C.c_double)),
        ("pi", C.POINTER(C.c_double)),
        ("normalise", C.c_int),
        ("reversible", C.c_int),
        ("n_categories", C.c_int),
        ("cat_rates", C.POINTER(C.c_double)),
        ("cat_weights", C.POINTER(C.c_double)),
        ("n_taxa", C.c_int),
        ("heights", C.POINTER(C.c_double)),
        ("parent", C.POINTER(C.c_int)),
        ("branch_rates", C.POINTER(C.c_double)),
        ("n_patterns", C.c_int),
        ("tips", C.POINTER(C.c_int)),
        ("pattern_weights", C.POINTER(C.c_double)),
        ("n_masks", C.c_int),
        ("masks", C.POINTER(C.c_ulonglong)),
        ("n_params", C.c_int),
        ("dQ", C.POINTER(C.c_double)),
        ("scaling", C.c_int),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        pp = C.POINTER(_Problem)
        _lib.or_normalise.restype = C.c_double
        _lib.or_normalise.argtypes = [C.c_int, dp, dp, dp]
        _lib.or_eig_sym.restype = C.c_int
        _lib.or_eig_sym.argtypes = [C.c_int, dp, dp, dp, dp, dp]
        _lib.or_expm.restype = C.c_int
        _lib.or_expm.argtypes = [C.c_int, dp, dp, C.c_int, C.c_double, dp]
        _lib.or_frechet.restype = C.c_int
        _lib.or_frechet.argtypes = [C.c_int, dp, dp, dp]
        _lib.or_segments.restype = C.c_int
        _lib.or_segments.argtypes = [C.c_int, dp, C.c_double, C.c_double, C.c_int,
                                     C.c_int, C.c_int, ip, dp, ip, ip]
        _lib.or_branch_matrix.restype = C.c_int
        _lib.or_branch_matrix.argtypes = [pp, C.c_int, C.c_int, dp]
        _lib.or_log_likelihood.restype = C.c_double
        _lib.or_log_likelihood.argtypes = [pp, dp]
        _lib.or_brute_force.restype = C.c_double
        _lib.or_brute_force.argtypes = [pp, dp]
        _lib.or_branch_adjoints.restype = C.c_int
        _lib.or_branch_adjoints.argtypes = [pp, dp, dp]
        _lib.or_gradient.restype = C.c_int
        _lib.or_gradient.argtypes = [pp, dp, dp, dp, dp, dp]
        _lib.or_expected_counts.restype = C.c_int
        _lib.or_expected_counts.argtypes = [pp, dp, dp]
        _lib.or_ancestral.restype = C.c_int
        _lib.or_ancestral.argtypes = [pp, dp]
        _lib.or_ancestral_brute.restype = C.c_int
        _lib.or_ancestral_brute.argtypes = [pp, dp]
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(C.POINTER(C.c_int))


class _Packed:
    """Holds the numpy buffers alive while the C struct points at them."""

    def __init__(self, w, scaling=True):
        keep = []

        def d(x):
            if x is None:
                return None
            a, p = _d(x)
            keep.append(a)
            return p

        def i(x):
            if x is None:
                return None
            a, p = _i(x)
            keep.append(a)
            return p

        K = int(w.K)
        Q = np.asarray(w.Q, dtype=np.float64).reshape(-1, K, K)
        S = Q.shape[0]
        E = int(w.n_epochs)
        tips = np.asarray(w.tips, dtype=np.int32)
        N = tips.shape[0]
        P = tips.shape[1]
        masks = getattr(w, "masks", None)
        dQ = getattr(w, "dQ", None)
        n_params = 0 if dQ is None else int(np.asarray(dQ).shape[0])
        pr = _Problem()
        pr.K = K
        pr.n_epochs = E
        pr.boundaries = d(np.asarray(w.boundaries, dtype=np.float64).reshape(-1)
                          if E > 1 else np.zeros(1))
        phi = getattr(w, "epoch_to_matrix", None)
        pr.epoch_to_matrix = i(phi) if phi is not None else None
        pr.n_matrices = S
        pr.Q = d(Q)
        pr.pi = d(w.pi)
        pr.normalise = int(getattr(w, "normalise", 1))
        pr.reversible = int(getattr(w, "reversible", 1))
        pr.n_categories = int(len(w.cat_rates))
        pr.cat_rates = d(w.cat_rates)
        pr.cat_weights = d(w.cat_weights)
        pr.n_taxa = N
        pr.heights = d(w.heights)
        pr.parent = i(w.parent)
        br = getattr(w, "branch_rates", None)
        pr.branch_rates = d(br) if br is not None else None
        pr.n_patterns = P
        pr.tips = i(tips)
        pr.pattern_weights = d(w.pattern_weights)
        if masks is not None and len(masks):
            m = np.ascontiguousarray(masks, dtype=np.uint64)
            keep.append(m)
            pr.n_masks = int(m.shape[0])
            pr.masks = m.ctypes.data_as(C.POINTER(C.c_ulonglong))
        else:
            pr.n_masks = 0
            pr.masks = None
        pr.n_params = n_params
        pr.dQ = d(dQ) if n_params else None
        pr.scaling = 1 if scaling else 0
        self.pr = pr
        self.keep = keep
        self.K, self.S, self.E, self.N, self.P = K, S, E, N, P
        self.C = pr.n_categories
        self.n_params = n_params


def log_likelihood(w, scaling=True):
    """lnL = sum_p n_p log sum_c w_c sum_i pi_i L_root(c,p,i) (Eq. partial_likelihood
    and the root sum that follows it).  Returns (lnL, per-pattern log-likelihoods)."""
    lib = _load()
    pk = _Packed(w, scaling)
    site = np.zeros(pk.P)
    val = lib.or_log_likelihood(C.byref(pk.pr), site.ctypes.data_as(C.POINTER(C.c_double)))
    return float(val), site


def brute_force(w):
    """lnL by explicit summation over every internal-node state assignment."""
    lib = _load()
    pk = _Packed(w, False)
    site = np.zeros(pk.P)
    val = lib.or_brute_force(C.byref(pk.pr), site.ctypes.data_as(C.POINTER(C.c_double)))
    return float(val), site


def branch_matrix(w, node, cat):
    """P(t_u, t_v, r_v) of the branch above ``node`` for category ``cat``
    (Eq. convolution, parent-end factor on the left)."""
    lib = _load()
    pk = _Packed(w)
    out = np.zeros((pk.K, pk.K))
    rc = lib.or_branch_matrix(C.byref(pk.pr), int(node), int(cat),
                              out.ctypes.data_as(C.POINTER(C.c_double)))
    if rc != 0:
        raise RuntimeError(f"oracle branch_matrix failed ({rc})")
    return out


def branch_adjoints(w, scaling=True):
    """G[v][c] = d lnL / d P_v,c for every non-root node v: (lnL, G[nodes][C][K][K])."""
    lib = _load()
    pk = _Packed(w, scaling)
    nn = 2 * pk.N - 1
    G = np.zeros((nn, pk.C, pk.K, pk.K))
    lnl = C.c_double(0.0)
    rc = lib.or_branch_adjoints(C.byref(pk.pr), G.ctypes.data_as(C.POINTER(C.c_double)),
                                C.byref(lnl))
    if rc != 0:
        raise RuntimeError(f"oracle branch_adjoints failed ({rc})")
    return lnl.value, G


def gradient(w, scaling=True):
    """Analytic gradient.  Returns dict with lnL and d/d heights [2N-1],
    d/d boundaries [E-1], d/d params [n_params], d/d branch rates [2N-1]."""
    lib = _load()
    pk = _Packed(w, scaling)
    nn = 2 * pk.N - 1
    dh = np.zeros(nn)
    db = np.zeros(max(pk.E - 1, 1))
    dp = np.zeros(max(pk.n_params, 1))
    dr = np.zeros(nn)
    lnl = C.c_double(0.0)
    P = C.POINTER(C.c_double)
    rc = lib.or_gradient(C.byref(pk.pr), C.byref(lnl), dh.ctypes.data_as(P),
                         db.ctypes.data_as(P), dp.ctypes.data_as(P), dr.ctypes.data_as(P))
    if rc != 0:
        raise RuntimeError(f"oracle gradient failed ({rc})")
    return {"lnL": lnl.value, "heights": dh, "boundaries": db[: pk.E - 1],
            "params": dp[: pk.n_params], "branch_rates": dr}


def expected_counts(w, scaling=True):
    """Expected numbers of i -> j transitions given the data, summed over the
    weighted patterns and the categories: per branch [2N-1][K][K] and per
    epoch [E][K][K] (q_ij times the derivative of lnL with respect to q_ij
    with q_ii held fixed, segment by segment; Minin and Suchard 2008)."""
    lib = _load()
    pk = _Packed(w, scaling)
    nn = 2 * pk.N - 1
    per_branch = np.zeros((nn, pk.K, pk.K))
    per_epoch = np.zeros((pk.E, pk.K, pk.K))
    P = C.POINTER(C.c_double)
    rc = lib.or_expected_counts(C.byref(pk.pr), per_branch.ctypes.data_as(P),
                                per_epoch.ctypes.data_as(P))
    if rc != 0:
        raise RuntimeError(f"oracle expected_counts failed ({rc})")
    return per_branch, per_epoch


def ancestral_states(w, brute=False):
    """Marginal posterior of every internal node's state given each pattern,
    [N-1][P][K] (internal nodes N..2N-2 in order): outside x inside
    probabilities summed over categories and normalised; ``brute=True``
    enumerates every joint assignment instead (small trees only)."""
    lib = _load()
    pk = _Packed(w, True)
    out = np.zeros((pk.N - 1, pk.P, pk.K))
    fn = lib.or_ancestral_brute if brute else lib.or_ancestral
    rc = fn(C.byref(pk.pr), out.ctypes.data_as(C.POINTER(C.c_double)))
    if rc != 0:
        raise RuntimeError(f"oracle ancestral states failed ({rc})")
    return out


def normalise(Q, pi):
    """Scale Q so that sum_i pi_i q_ii = -1 (Methods).  Returns (Qn, c)."""
    lib = _load()
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    K = Q.shape[0]
    out = np.zeros_like(Q)
    pia = np.ascontiguousarray(pi, dtype=np.float64)
    c = lib.or_normalise(K, _d(Q)[1], pia.ctypes.data_as(C.POINTER(C.c_double)),
                         out.ctypes.data_as(C.POINTER(C.c_double)))
    return out, c


def eig_sym(Q, pi):
    """(lambda, V, Vinv) with Q = V diag(lambda) Vinv for reversible Q."""
    lib = _load()
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    K = Q.shape[0]
    lam = np.zeros(K)
    V = np.zeros((K, K))
    Vi = np.zeros((K, K))
    pia = np.ascontiguousarray(pi, dtype=np.float64)
    P = C.POINTER(C.c_double)
    rc = lib.or_eig_sym(K, Q.ctypes.data_as(P), pia.ctypes.data_as(P), lam.ctypes.data_as(P),
                        V.ctypes.data_as(P), Vi.ctypes.data_as(P))
    if rc < 0:
        raise RuntimeError("oracle Jacobi did not converge")
    return lam, V, Vi


def expm(Q, tau, pi=None, reversible=True):
    """exp(tau Q): eigen path (reversible, needs pi) or uniformisation."""
    lib = _load()
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    K = Q.shape[0]
    out = np.zeros((K, K))
    pia = np.ascontiguousarray(pi if pi is not None else np.full(K, 1.0 / K), dtype=np.float64)
    P = C.POINTER(C.c_double)
    rc = lib.or_expm(K, Q.ctypes.data_as(P), pia.ctypes.data_as(P), 1 if reversible else 0,
                     float(tau), out.ctypes.data_as(P))
    if rc != 0:
        raise RuntimeError("oracle expm failed")
    return out


def frechet(X, Y):
    """Frechet derivative of exp at X in direction Y (block-triangular exp)."""
    lib = _load()
    X = np.ascontiguousarray(X, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    K = X.shape[0]
    out = np.zeros((K, K))
    P = C.POINTER(C.c_double)
    lib.or_frechet(K, X.ctypes.data_as(P), Y.ctypes.data_as(P), out.ctypes.data_as(P))
    return out


def segments(boundaries, h_child, h_parent, parent=-1, child=-1):
    """Epoch segments of one branch, parent end first:
    list of (epoch, dt, hi_ref, lo_ref); refs are node ids or -(j+1) for boundary j."""
    lib = _load()
    b = np.ascontiguousarray(boundaries, dtype=np.float64).reshape(-1)
    E = b.shape[0] + 1
    ep = np.zeros(64, dtype=np.int32)
    dt = np.zeros(64)
    hi = np.zeros(64, dtype=np.int32)
    lo = np.zeros(64, dtype=np.int32)
    bb = b if b.size else np.zeros(1)
    n = lib.or_segments(E, bb.ctypes.data_as(C.POINTER(C.c_double)), float(h_child),
                        float(h_parent), int(parent), int(child), 64,
                        ep.ctypes.data_as(C.POINTER(C.c_int)), dt.ctypes.data_as(C.POINTER(C.c_double)),
                        hi.ctypes.data_as(C.POINTER(C.c_int)), lo.ctypes.data_as(C.POINTER(C.c_int)))
    if n < 0:
        raise RuntimeError("too many segments")
    return [(int(ep[k]), float(dt[k]), int(hi[k]), int(lo[k])) for k in range(n)]
