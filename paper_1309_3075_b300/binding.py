"""ctypes binding of libepoch (include/epoch.h): argument marshalling only.

Every function below has the name of the C entry point it calls and does
nothing but convert numpy / torch arguments to pointers and raise on a
non-zero status.  All arithmetic of the likelihood path runs in the CUDA
kernels of libepoch.so; there is no CPU fallback: if the library cannot be
loaded, importing this module's functions raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libepoch.so")

EPOCH_FP64, EPOCH_FP32, EPOCH_FP32_TC, EPOCH_FP32_AUTO, EPOCH_FP32_TC_BF16 = 0, 1, 2, 3, 4
STATUS = {0: "EPOCH_OK", 1: "EPOCH_ERR_ARG", 2: "EPOCH_ERR_ORDER", 3: "EPOCH_ERR_CAPACITY",
          4: "EPOCH_ERR_NUMERIC", 5: "EPOCH_ERR_CUDA", 6: "EPOCH_ERR_TIMEOUT",
          7: "EPOCH_ERR_UNSUPPORTED"}


class EpochError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} {msg}".strip())


_lib = None
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_vp = C.c_void_p

# name -> argtypes (restype is int status unless listed in _RESTYPE)
_SIGS = {
    "epoch_create": [C.POINTER(_vp), C.c_int, C.c_int, _dp, _ip, C.c_int, C.c_int, C.c_int,
                     C.c_int, C.c_int, _vp],
    "epoch_destroy": [_vp],
    "epoch_last_error": [_vp],
    "epoch_path_info": [_vp, _ip, _dp, _dp, _dp],
    # addresses as plain integers: the step is called every iteration, and
    # an int marshals several times faster than a typed pointer
    "epoch_evaluate_step": [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, C.c_int, _dp, _vp, _vp, _vp,
                            _vp],
    "epoch_status_string": [C.c_int],
    "epoch_set_boundaries": [_vp, _dp],
    "epoch_set_rate_matrices": [_vp, _dp, _dp, C.c_int, C.c_int],
    "epoch_set_rate_derivatives": [_vp, C.c_int, _dp],
    "epoch_set_categories": [_vp, _dp, _dp],
    "epoch_set_ambiguity_masks": [_vp, C.c_int, C.POINTER(C.c_ulonglong)],
    "epoch_set_tree": [_vp, C.c_int, _dp, _ip, _dp],
    "epoch_check_tree": [C.c_int, _dp, _ip, _dp, _ip],
    "epoch_set_heights": [_vp, _dp],
    "epoch_set_tip_data": [_vp, _ip, _dp],
    "epoch_compute_branch_matrices": [_vp],
    "epoch_update_partials": [_vp],
    "epoch_log_likelihood": [_vp, _dp],
    "epoch_site_log_likelihoods": [_vp, _dp],
    "epoch_gradient": [_vp, _dp, _dp, _dp, _dp],
    "epoch_get_branch_matrix": [_vp, C.c_int, C.c_int, _dp],
    "epoch_expected_counts": [_vp, _dp, _dp],
    "epoch_ancestral_states": [_vp, _dp],
    "epoch_evaluate_async": [_vp, C.c_int],
    "epoch_read_results": [_vp, _dp, _dp, _dp, _dp, _dp],
    "epoch_counters": [_vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)],
    "epoch_set_heights_device": [_vp, _vp],
    "epoch_read_results_device": [_vp, _vp, _vp],
    "epoch_site_log_sum_noalloc": [_vp, _vp, C.c_int, C.c_longlong, _vp, C.c_int, _vp, _vp,
                                   _vp],
    "epoch_batch_create": [C.POINTER(_vp), C.c_int, C.c_int, _ip, _ip, _ip, _vp],
    "epoch_batch_destroy": [_vp],
    "epoch_batch_last_error": [_vp],
    "epoch_batch_set_models": [_vp, _dp, _dp, _dp, C.c_int],
    "epoch_batch_set_trees": [_vp, _dp, _ip],
    "epoch_batch_set_tip_data": [_vp, _ip, _dp],
    "epoch_batch_evaluate_async": [_vp],
    "epoch_batch_read": [_vp, _dp],
    "epoch_batch_launch_shape": [_vp, _ip, _ip],
    "epoch_batch_evaluate_gradient_async": [_vp],
    "epoch_batch_read_gradient": [_vp, _dp, _dp, _dp],
}
_RESTYPE = {"epoch_destroy": None, "epoch_last_error": C.c_char_p,
            "epoch_status_string": C.c_char_p, "epoch_batch_destroy": None,
            "epoch_batch_last_error": C.c_char_p}


def lib():
    """Load libepoch.so (built by paper_1309_3075_b300/build.py).  Raises if
    it is missing: the package has no other implementation."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libepoch.so not built ({LIB_PATH}); run "
                               "python -m paper_1309_3075_b300.build")
        L = C.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = _RESTYPE.get(name, C.c_int)
        _lib = L
    return _lib


def declared_symbols():
    return list(_SIGS)


def _d(a):
    if a is None:
        return None, None
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _i(a):
    if a is None:
        return None, None
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_ip)


def _check(ctx, st, where):
    if st != 0:
        msg = lib().epoch_last_error(ctx).decode() if ctx else ""
        raise EpochError(st, where, msg)


# ---- thin wrappers with the C names ----------------------------------------

def epoch_create(states, n_epochs, boundaries, epoch_to_matrix, n_matrices, max_taxa,
                 n_patterns, n_categories, precision=EPOCH_FP32, cuda_stream=None):
    out = _vp()
    b, bp = _d(boundaries if n_epochs > 1 else None)
    phi, php = _i(epoch_to_matrix)
    st = lib().epoch_create(C.byref(out), int(states), int(n_epochs), bp, php, int(n_matrices),
                            int(max_taxa), int(n_patterns), int(n_categories), int(precision),
                            _vp(cuda_stream) if cuda_stream else None)
    _check(None, st, "epoch_create")
    return out


def epoch_destroy(ctx):
    lib().epoch_destroy(ctx)


def epoch_set_boundaries(ctx, boundaries):
    b, bp = _d(boundaries)
    _check(ctx, lib().epoch_set_boundaries(ctx, bp), "epoch_set_boundaries")


def epoch_set_rate_matrices(ctx, Q, pi, normalise=1, reversible=1):
    q, qp = _d(Q)
    p, pp = _d(pi)
    _check(ctx, lib().epoch_set_rate_matrices(ctx, qp, pp, int(normalise), int(reversible)),
           "epoch_set_rate_matrices")


def epoch_set_rate_derivatives(ctx, dQ):
    n = 0 if dQ is None else int(np.asarray(dQ).shape[0])
    q, qp = _d(dQ if n else None)
    _check(ctx, lib().epoch_set_rate_derivatives(ctx, n, qp), "epoch_set_rate_derivatives")


def epoch_set_categories(ctx, rates, weights):
    r, rp = _d(rates)
    w, wp = _d(weights)
    _check(ctx, lib().epoch_set_categories(ctx, rp, wp), "epoch_set_categories")


def epoch_set_ambiguity_masks(ctx, masks):
    m = np.ascontiguousarray(masks if masks is not None else [], dtype=np.uint64)
    ptr = m.ctypes.data_as(C.POINTER(C.c_ulonglong)) if m.size else None
    _check(ctx, lib().epoch_set_ambiguity_masks(ctx, int(m.size), ptr), "epoch_set_ambiguity_masks")


def epoch_set_tree(ctx, heights, parent, branch_rates=None):
    h, hp = _d(heights)
    p, pp = _i(parent)
    r, rp = _d(branch_rates)
    n_taxa = (len(h) + 1) // 2
    _check(ctx, lib().epoch_set_tree(ctx, n_taxa, hp, pp, rp), "epoch_set_tree")


def epoch_check_tree(heights, parent, branch_rates=None):
    """Returns (status, n_levels); runs on the host only."""
    h, hp = _d(heights)
    p, pp = _i(parent)
    r, rp = _d(branch_rates)
    nl = C.c_int(-1)
    st = lib().epoch_check_tree((len(h) + 1) // 2, hp, pp, rp, C.byref(nl))
    return st, nl.value


def epoch_set_heights(ctx, heights):
    h, hp = _d(heights)
    _check(ctx, lib().epoch_set_heights(ctx, hp), "epoch_set_heights")


def epoch_set_tip_data(ctx, tip_codes, pattern_weights):
    t, tp = _i(tip_codes)
    w, wp = _d(pattern_weights)
    _check(ctx, lib().epoch_set_tip_data(ctx, tp, wp), "epoch_set_tip_data")


def epoch_compute_branch_matrices(ctx):
    _check(ctx, lib().epoch_compute_branch_matrices(ctx), "epoch_compute_branch_matrices")


def epoch_update_partials(ctx):
    _check(ctx, lib().epoch_update_partials(ctx), "epoch_update_partials")


def epoch_log_likelihood(ctx):
    out = C.c_double(0.0)
    _check(ctx, lib().epoch_log_likelihood(ctx, C.byref(out)), "epoch_log_likelihood")
    return out.value


def epoch_site_log_likelihoods(ctx, n_patterns):
    out = np.zeros(n_patterns)
    _check(ctx, lib().epoch_site_log_likelihoods(ctx, out.ctypes.data_as(_dp)),
           "epoch_site_log_likelihoods")
    return out


def epoch_gradient(ctx, n_nodes, n_epochs, n_params):
    dh = np.zeros(n_nodes)
    db = np.zeros(max(n_epochs - 1, 1))
    dp = np.zeros(max(n_params, 1))
    dr = np.zeros(n_nodes)
    _check(ctx, lib().epoch_gradient(ctx, dh.ctypes.data_as(_dp), db.ctypes.data_as(_dp),
                                     dp.ctypes.data_as(_dp) if n_params else None,
                                     dr.ctypes.data_as(_dp)), "epoch_gradient")
    return {"heights": dh, "boundaries": db[: n_epochs - 1], "params": dp[:n_params],
            "branch_rates": dr}


def epoch_expected_counts(ctx, n_nodes, n_epochs, K):
    """Expected transition counts of the last gradient evaluation:
    (per_branch [n_nodes][K][K], per_epoch [n_epochs][K][K])."""
    per_branch = np.zeros((n_nodes, K, K))
    per_epoch = np.zeros((n_epochs, K, K))
    _check(ctx, lib().epoch_expected_counts(ctx, per_branch.ctypes.data_as(_dp),
                                            per_epoch.ctypes.data_as(_dp)),
           "epoch_expected_counts")
    return per_branch, per_epoch


def epoch_ancestral_states(ctx, n_taxa, n_patterns, K):
    """Posterior state probabilities of the internal nodes, [N-1][P][K]."""
    out = np.zeros((n_taxa - 1, n_patterns, K))
    _check(ctx, lib().epoch_ancestral_states(ctx, out.ctypes.data_as(_dp)),
           "epoch_ancestral_states")
    return out


def epoch_get_branch_matrix(ctx, node, category, K):
    out = np.zeros((K, K))
    _check(ctx, lib().epoch_get_branch_matrix(ctx, int(node), int(category),
                                              out.ctypes.data_as(_dp)), "epoch_get_branch_matrix")
    return out


def epoch_evaluate_async(ctx, with_gradient=True):
    _check(ctx, lib().epoch_evaluate_async(ctx, 1 if with_gradient else 0), "epoch_evaluate_async")


def epoch_read_results(ctx, n_nodes=0, n_epochs=1, n_params=0, with_gradient=True):
    lnl = C.c_double(0.0)
    if not with_gradient:
        _check(ctx, lib().epoch_read_results(ctx, C.byref(lnl), None, None, None, None),
               "epoch_read_results")
        return lnl.value, None
    dh = np.zeros(n_nodes)
    db = np.zeros(max(n_epochs - 1, 1))
    dp = np.zeros(max(n_params, 1))
    dr = np.zeros(n_nodes)
    _check(ctx, lib().epoch_read_results(ctx, C.byref(lnl), dh.ctypes.data_as(_dp),
                                         db.ctypes.data_as(_dp),
                                         dp.ctypes.data_as(_dp) if n_params else None,
                                         dr.ctypes.data_as(_dp)), "epoch_read_results")
    return lnl.value, {"heights": dh, "boundaries": db[: n_epochs - 1], "params": dp[:n_params],
                       "branch_rates": dr}


def epoch_set_heights_device(ctx, heights_ptr):
    """heights_ptr: device address (int) of 2N-1 float64 values."""
    _check(ctx, lib().epoch_set_heights_device(ctx, _vp(int(heights_ptr))),
           "epoch_set_heights_device")


def epoch_read_results_device(ctx, lnl_ptr=0, grad_ptr=0):
    """Device addresses (int, 0 = not wanted); async on the context's stream."""
    _check(ctx, lib().epoch_read_results_device(ctx, _vp(int(lnl_ptr)) if lnl_ptr else None,
                                                _vp(int(grad_ptr)) if grad_ptr else None),
           "epoch_read_results_device")


_F64 = np.dtype(np.float64)


def _opt(a):
    """The address of an array already float64 and contiguous (the caller's
    buffer, no copy), or NULL for None."""
    if a is None:
        return None
    if a.dtype != _F64 or not a.flags.c_contiguous:
        raise ValueError("step inputs must be contiguous float64 arrays")
    return a.ctypes.data


_STEP_OUT = ("heights", "boundaries", "params", "branch_rates")


def epoch_evaluate_step(ctx, Q=None, pi=None, dQ=None, boundaries=None, cat_rates=None,
                        cat_weights=None, heights=None, with_gradient=True, out=None):
    """One inference step in one call (see include/epoch.h).  Inputs and the
    outputs in ``out`` (a dict of preallocated float64 arrays with keys
    heights, boundaries, params, branch_rates) are passed without copies.
    Returns lnL."""
    lnl = C.c_double(0.0)
    o = out or {}
    _check(ctx, lib().epoch_evaluate_step(
        ctx, _opt(Q), _opt(pi), _opt(dQ), _opt(boundaries), _opt(cat_rates), _opt(cat_weights),
        _opt(heights), 1 if with_gradient else 0, C.byref(lnl),
        *[_opt(o.get(k)) for k in _STEP_OUT]),
        "epoch_evaluate_step")
    return lnl.value


def epoch_step_function(ctx, Q=None, pi=None, dQ=None, boundaries=None, cat_rates=None,
                        cat_weights=None, heights=None, with_gradient=True, out=None):
    """epoch_evaluate_step bound to fixed buffers: the arrays' addresses are
    taken once, and the returned function (no arguments, returns lnL) makes
    the call with them.  The caller updates the input arrays in place
    between calls and reads the gradient from ``out``; the arrays must stay
    alive (and not be resized) while the function is in use."""
    o = out or {}
    arrays = [Q, pi, dQ, boundaries, cat_rates, cat_weights, heights] + [o.get(k) for k in _STEP_OUT]
    addr = [_opt(a) for a in arrays]
    lnl = C.c_double(0.0)
    args = (ctx, *addr[:7], 1 if with_gradient else 0, C.byref(lnl), *addr[7:])
    fn = lib().epoch_evaluate_step

    def step():
        st = fn(*args)
        if st != 0:
            _check(ctx, st, "epoch_evaluate_step")
        return lnl.value

    step.buffers = arrays  # keeps the arrays referenced
    return step


def epoch_path_info(ctx):
    """(precision in use, probe ms SIMT, probe ms TF32 x 3, probe ms BF16 x 3)."""
    p, a, b, e = C.c_int(0), C.c_double(0.0), C.c_double(0.0), C.c_double(0.0)
    _check(ctx, lib().epoch_path_info(ctx, C.byref(p), C.byref(a), C.byref(b), C.byref(e)),
           "epoch_path_info")
    return p.value, a.value, b.value, e.value


def epoch_counters(ctx):
    a, b = C.c_longlong(0), C.c_longlong(0)
    _check(ctx, lib().epoch_counters(ctx, C.byref(a), C.byref(b)), "epoch_counters")
    return a.value, b.value


# ---- convenience: one context for one workload-shaped problem ---------------

class EpochLikelihood:
    """Owns one libepoch context.  ``w`` is any object with the attributes of
    ``synth.Workload`` (K, boundaries, epoch_to_matrix, Q, pi, normalise,
    reversible, cat_rates, cat_weights, heights, parent, branch_rates, tips,
    pattern_weights, masks, dQ).  Methods call the C entry points in order."""

    def __init__(self, w, precision=EPOCH_FP32, max_taxa=None, cuda_stream=None):
        self.K = int(w.K)
        self.E = len(np.asarray(w.boundaries).reshape(-1)) + 1
        self.S = int(np.asarray(w.Q).shape[0])
        self.N = int(np.asarray(w.tips).shape[0])
        self.P = int(np.asarray(w.tips).shape[1])
        self.C = int(len(w.cat_rates))
        self.precision = precision
        self.cuda_stream = cuda_stream
        phi = getattr(w, "epoch_to_matrix", None)
        self.ctx = epoch_create(self.K, self.E, w.boundaries, phi, self.S,
                                max_taxa or self.N, self.P, self.C, precision, cuda_stream)
        self.path = epoch_path_info(self.ctx)[0]  # EPOCH_FP32_AUTO resolved
        self.n_params = 0
        self.load(w)

    def load(self, w, tips=True):
        ctx = self.ctx
        masks = getattr(w, "masks", None)
        if masks is not None and len(masks):
            epoch_set_ambiguity_masks(ctx, masks)
        if self.E > 1:
            epoch_set_boundaries(ctx, w.boundaries)
        epoch_set_rate_matrices(ctx, w.Q, w.pi, getattr(w, "normalise", 1),
                                getattr(w, "reversible", 1))
        dQ = getattr(w, "dQ", None)
        if dQ is not None and int(getattr(w, "reversible", 1)):
            epoch_set_rate_derivatives(ctx, dQ)
            self.n_params = int(np.asarray(dQ).shape[0])
        else:
            epoch_set_rate_derivatives(ctx, None)
            self.n_params = 0
        epoch_set_categories(ctx, w.cat_rates, w.cat_weights)
        epoch_set_tree(ctx, w.heights, w.parent, getattr(w, "branch_rates", None))
        if tips:
            epoch_set_tip_data(ctx, w.tips, w.pattern_weights)

    def log_likelihood(self):
        epoch_compute_branch_matrices(self.ctx)
        epoch_update_partials(self.ctx)
        return epoch_log_likelihood(self.ctx)

    def site_log_likelihoods(self):
        return epoch_site_log_likelihoods(self.ctx, self.P)

    def gradient(self):
        return epoch_gradient(self.ctx, 2 * self.N - 1, self.E, self.n_params)

    def branch_matrix(self, node, cat):
        return epoch_get_branch_matrix(self.ctx, node, cat, self.K)

    def expected_counts(self):
        """(per_branch, per_epoch) expected i -> j transition counts of the
        last gradient evaluation."""
        return epoch_expected_counts(self.ctx, 2 * self.N - 1, self.E, self.K)

    def ancestral_states(self):
        """Posterior state probabilities of the internal nodes [N-1][P][K]
        (the last gradient evaluation)."""
        return epoch_ancestral_states(self.ctx, self.N, self.P, self.K)

    def evaluate(self, with_gradient=True):
        epoch_evaluate_async(self.ctx, with_gradient)
        return epoch_read_results(self.ctx, 2 * self.N - 1, self.E, self.n_params, with_gradient)

    def counters(self):
        return epoch_counters(self.ctx)

    def close(self):
        if self.ctx:
            epoch_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def epoch_site_log_sum_noalloc(site_log, exponents, n_rows, row_stride, weights, n_patterns,
                               site_out, lnl_out, cuda_stream=None):
    """Device-pointer call (integers, e.g. ``tensor.data_ptr()``; 0 or None for
    NULL).  Returns the status code instead of raising, so callers can see
    EPOCH_ERR_CAPACITY; the call allocates no device memory."""
    def p(x):
        return _vp(int(x)) if x else None
    return int(lib().epoch_site_log_sum_noalloc(p(site_log), p(exponents), int(n_rows),
                                                int(row_stride), p(weights), int(n_patterns),
                                                p(site_out), p(lnl_out), p(cuda_stream)))


# ---- many trees in one launch ------------------------------------------------

def _bcheck(b, st, where):
    if st != 0:
        msg = lib().epoch_batch_last_error(b).decode() if b else ""
        raise EpochError(st, where, msg)


def epoch_batch_create(states, n_taxa, n_epochs, n_patterns, cuda_stream=None):
    out = _vp()
    nt, ntp = _i(n_taxa)
    ne, nep = _i(n_epochs)
    npt, npp = _i(n_patterns)
    st = lib().epoch_batch_create(C.byref(out), int(states), len(nt), ntp, nep, npp,
                                  _vp(cuda_stream) if cuda_stream else None)
    _bcheck(None, st, "epoch_batch_create")
    return out


def epoch_batch_destroy(b):
    lib().epoch_batch_destroy(b)


def epoch_batch_set_models(b, boundaries, Q, pi, normalise=1):
    bd, bdp = _d(boundaries)
    q, qp = _d(Q)
    p, pp = _d(pi)
    _bcheck(b, lib().epoch_batch_set_models(b, bdp if bd is not None and bd.size else None, qp,
                                            pp, int(normalise)), "epoch_batch_set_models")


def epoch_batch_set_trees(b, heights, parent):
    h, hp = _d(heights)
    p, pp = _i(parent)
    _bcheck(b, lib().epoch_batch_set_trees(b, hp, pp), "epoch_batch_set_trees")


def epoch_batch_set_tip_data(b, codes, weights):
    c, cp = _i(codes)
    w, wp = _d(weights)
    _bcheck(b, lib().epoch_batch_set_tip_data(b, cp, wp), "epoch_batch_set_tip_data")


def epoch_batch_evaluate_async(b):
    _bcheck(b, lib().epoch_batch_evaluate_async(b), "epoch_batch_evaluate_async")


def epoch_batch_read(b, n_trees):
    out = np.zeros(n_trees)
    _bcheck(b, lib().epoch_batch_read(b, out.ctypes.data_as(_dp)), "epoch_batch_read")
    return out


def epoch_batch_evaluate_gradient_async(b):
    _bcheck(b, lib().epoch_batch_evaluate_gradient_async(b), "epoch_batch_evaluate_gradient_async")


def epoch_batch_read_gradient(b, n_trees, n_nodes, n_boundaries):
    lnl = np.empty(n_trees)
    dh = np.empty(n_nodes)
    db = np.empty(max(n_boundaries, 1))
    _bcheck(b, lib().epoch_batch_read_gradient(b, lnl.ctypes.data_as(_dp), dh.ctypes.data_as(_dp),
                                               db.ctypes.data_as(_dp) if n_boundaries else None),
            "epoch_batch_read_gradient")
    return lnl, dh, db[:n_boundaries]


def epoch_batch_launch_shape(b):
    w, c = C.c_int(0), C.c_int(0)
    _bcheck(b, lib().epoch_batch_launch_shape(b, C.byref(w), C.byref(c)),
            "epoch_batch_launch_shape")
    return w.value, c.value


class EpochBatch:
    """Owns one epoch_batch.  ``trees`` is a sequence of objects with the
    attributes of ``synth.Workload`` (one rate matrix per epoch, one
    category, at most 4 patterns); arrays are concatenated in tree order."""

    def __init__(self, trees, cuda_stream=None):
        trees = list(trees)
        self.T = len(trees)
        self.K = int(trees[0].K)
        self._nodes = [2 * np.asarray(t.tips).shape[0] - 1 for t in trees]
        self._bnds = [len(np.asarray(t.boundaries).reshape(-1)) for t in trees]
        self.b = epoch_batch_create(
            self.K, [np.asarray(t.tips).shape[0] for t in trees],
            [len(np.asarray(t.boundaries).reshape(-1)) + 1 for t in trees],
            [np.asarray(t.tips).shape[1] for t in trees], cuda_stream)
        self.load(trees)

    def load(self, trees):
        bnd = np.concatenate([np.asarray(t.boundaries, dtype=np.float64).reshape(-1)
                              for t in trees])
        Q = np.concatenate([np.asarray(t.Q, dtype=np.float64).reshape(-1) for t in trees])
        pi = np.concatenate([np.asarray(t.pi, dtype=np.float64).reshape(-1) for t in trees])
        epoch_batch_set_models(self.b, bnd, Q, pi, int(getattr(trees[0], "normalise", 1)))
        epoch_batch_set_trees(self.b, np.concatenate([np.asarray(t.heights) for t in trees]),
                              np.concatenate([np.asarray(t.parent) for t in trees]))
        epoch_batch_set_tip_data(self.b,
                                 np.concatenate([np.asarray(t.tips).reshape(-1) for t in trees]),
                                 np.concatenate([np.asarray(t.pattern_weights, dtype=np.float64)
                                                 for t in trees]))

    def evaluate(self):
        epoch_batch_evaluate_async(self.b)
        return epoch_batch_read(self.b, self.T)

    def evaluate_gradient(self):
        """lnL per tree and, per tree, d lnL / d heights [2N_t - 1] and
        d lnL / d boundaries [E_t - 1] (lists of arrays)."""
        epoch_batch_evaluate_gradient_async(self.b)
        lnl, dh, db = epoch_batch_read_gradient(self.b, self.T, int(sum(self._nodes)),
                                                int(sum(self._bnds)))
        ho = np.cumsum([0] + self._nodes)
        bo = np.cumsum([0] + self._bnds)
        return (lnl, [dh[ho[t]:ho[t + 1]] for t in range(self.T)],
                [db[bo[t]:bo[t + 1]] for t in range(self.T)])

    def launch_shape(self):
        return epoch_batch_launch_shape(self.b)

    def close(self):
        if self.b:
            epoch_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
