"""CPU-side checks of the C ABI: the library loads, exports every entry point
include/*.h declares, validates arguments on the host before touching a
device, and has no CPU fallback (without a GPU, creating a context fails
with EPOCH_ERR_CUDA instead of computing anything)."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

import synth
from paper_1309_3075_b300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1309_3075_b300 import build

    build.build()
    return binding.lib()


def declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(epoch_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(L):
    names = declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
        assert n in binding.declared_symbols(), f"binding lacks {n}"


def test_status_strings(L):
    for s in range(8):
        assert L.epoch_status_string(s)


def test_create_rejects_bad_arguments_on_host(L):
    out = C.c_void_p()
    b = (C.c_double * 2)(0.3, 0.2)  # not increasing
    bad = [
        (1, 2, None, None, 2, 10, 10, 1, 1),       # K < 2
        (65, 1, None, None, 1, 10, 10, 1, 1),      # K > 64
        (4, 3, b, None, 3, 10, 10, 1, 1),          # unsorted boundaries
        (4, 1, None, None, 2, 10, 10, 1, 1),       # S != E without phi
        (4, 1, None, None, 1, 1, 10, 1, 1),        # max_taxa < 2
        (4, 1, None, None, 1, 10, 0, 1, 1),        # no patterns
        (4, 1, None, None, 1, 10, 10, 0, 1),       # no categories
        (4, 1, None, None, 1, 10, 10, 1, 7),       # unknown precision
    ]
    for args in bad:
        K, E, bnd, phi, S, N, P, Cc, prec = args
        st = L.epoch_create(C.byref(out), K, E, C.cast(bnd, C.POINTER(C.c_double)) if bnd else None,
                            phi, S, N, P, Cc, prec, None)
        assert st == 1, args
        assert not out.value


def test_no_cpu_fallback_without_gpu(L):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    out = C.c_void_p()
    st = L.epoch_create(C.byref(out), 4, 1, None, None, 1, 8, 16, 1, 1, None)
    assert st == 5  # EPOCH_ERR_CUDA: nothing computes without the device
    assert not out.value


def test_check_tree_host_validation(L):
    rng = np.random.default_rng(0)
    h, p = synth.coalescent_tree(20, rng)
    st, nl = binding.epoch_check_tree(h, p)
    assert st == 0 and nl >= 5
    # level count of a caterpillar is N-1
    N = 6
    hc = np.concatenate([np.zeros(N), np.arange(1, N)])
    pc = np.array([N, N] + [N + k for k in range(1, N - 1)] + list(range(N + 1, 2 * N - 1)) + [-1],
                  dtype=np.int32)
    assert binding.epoch_check_tree(hc, pc)[0] == 0
    assert binding.epoch_check_tree(hc, pc)[1] == N - 1
    p2 = p.copy()
    p2[3] = 3 + 0  # tip pointing at a tip
    assert binding.epoch_check_tree(h, p2)[0] == 1
    h2 = h.copy()
    h2[p[0]] = -1.0  # parent younger than child
    assert binding.epoch_check_tree(h2, p)[0] == 1
    p3 = p.copy()
    root = int(np.where(p < 0)[0][0])
    p3[root] = p[0]  # root gets a parent: a cycle and no root
    assert binding.epoch_check_tree(h, p3)[0] == 1
    r = np.ones(len(h))
    r[2] = np.nan
    assert binding.epoch_check_tree(h, p, r)[0] == 1
    p4 = p.copy()
    p4[0] = p[1] if p[1] != p[0] else p[2]  # a node with three children
    assert binding.epoch_check_tree(h, p4)[0] == 1


def test_build_flags_target_sm_103a():
    from paper_1309_3075_b300 import build

    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_step_call_marshals_without_copies_and_checks_its_arrays(L):
    """epoch_evaluate_step / epoch_step_function take contiguous float64 arrays
    by address (no copy): anything else is refused in the binding, and a NULL
    context is refused by the library before any device work."""
    ok = np.zeros(16)
    with pytest.raises(ValueError):
        binding.epoch_evaluate_step(None, Q=np.zeros(16, dtype=np.float32), pi=ok)
    with pytest.raises(ValueError):
        binding.epoch_step_function(None, heights=np.zeros((4, 4))[:, 1])
    with pytest.raises(binding.EpochError) as e:
        binding.epoch_evaluate_step(None, heights=ok)
    assert e.value.status == 1  # EPOCH_ERR_ARG
    buf = np.zeros(7)
    step = binding.epoch_step_function(None, heights=buf)
    assert step.buffers[6] is buf  # the caller's array itself, kept referenced
    with pytest.raises(binding.EpochError):
        step()
