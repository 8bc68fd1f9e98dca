"""epoch_site_log_sum_noalloc: the allocation-free weighted log-sum of the root
step, called through the C ABI with device pointers, against the
context-based entry points (epoch_log_likelihood, epoch_site_log_likelihoods)
and against a plain host sum of the same inputs.  Named to be collected last;
it also passes alone in a fresh process."""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

MAX_PATTERNS = 262144  # EPOCH_NOALLOC_MAX_PATTERNS in include/epoch.h


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    torch.cuda.set_device(0)
    return torch


def _existing(w):
    from paper_1309_3075_b300.binding import EPOCH_FP32, EpochLikelihood
    lik = EpochLikelihood(w, precision=EPOCH_FP32)
    try:
        lnl = lik.log_likelihood()
        site = np.asarray(lik.site_log_likelihoods(), dtype=np.float64)
    finally:
        lik.close()
    return lnl, site


def test_noalloc_matches_context_entry_points(torch_cuda):
    torch = torch_cuda
    from paper_1309_3075_b300.binding import epoch_site_log_sum_noalloc
    w = synth.small_nucleotide(4242, n_taxa=24, n_sites=700, n_cat=4, n_epochs=3, dated=True)
    lnl_ref, site_ref = _existing(w)
    P = site_ref.shape[0]
    dev = torch.device("cuda", 0)
    d_site = torch.tensor(site_ref, dtype=torch.float64, device=dev)
    d_w = torch.tensor(np.asarray(w.pattern_weights, dtype=np.float64), device=dev)
    d_out = torch.full((P,), float("nan"), dtype=torch.float64, device=dev)
    d_lnl = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):  # the second call checks that the counter was reset
        d_lnl.fill_(float("nan"))
        st = epoch_site_log_sum_noalloc(d_site.data_ptr(), 0, 0, 0, d_w.data_ptr(), P,
                                        d_out.data_ptr(), d_lnl.data_ptr(), stream)
        assert st == 0, st
        torch.cuda.synchronize()
        got = float(d_lnl.item())
        assert abs(got - lnl_ref) <= 1e-12 * abs(lnl_ref), (call, got, lnl_ref)
        np.testing.assert_allclose(d_out.cpu().numpy(), site_ref, rtol=0, atol=0)


def test_noalloc_exponents_and_no_growth(torch_cuda):
    torch = torch_cuda
    from paper_1309_3075_b300.binding import epoch_site_log_sum_noalloc
    rng = np.random.default_rng(77)
    P, rows, stride = 1000, 7, 1008
    site_log = rng.normal(-3.0, 1.0, P)
    ex = np.zeros((rows, stride), dtype=np.int16)
    ex[:, :P] = rng.integers(-40, 2, (rows, P))
    wts = rng.integers(0, 5, P).astype(np.float64)  # zero weights are skipped
    want_site = site_log + math.log(2.0) * ex[:, :P].astype(np.float64).sum(axis=0)
    want = math.fsum(float(a) * float(b) for a, b in zip(wts, want_site) if a != 0.0)
    dev = torch.device("cuda", 0)
    d_site = torch.tensor(site_log, device=dev)
    d_ex = torch.tensor(ex, device=dev)
    d_w = torch.tensor(wts, device=dev)
    d_out = torch.empty(P, dtype=torch.float64, device=dev)
    d_lnl = torch.empty(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    args = (d_site.data_ptr(), d_ex.data_ptr(), rows, stride, d_w.data_ptr(), P,
            d_out.data_ptr(), d_lnl.data_ptr(), stream)
    for _ in range(2):
        assert epoch_site_log_sum_noalloc(*args) == 0
        torch.cuda.synchronize()
        assert abs(float(d_lnl.item()) - want) <= 1e-12 * abs(want)
        np.testing.assert_allclose(d_out.cpu().numpy(), want_site, rtol=1e-15, atol=1e-12)
    # after the first call has set up the scratch, further calls leave the
    # device's free memory unchanged
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert epoch_site_log_sum_noalloc(*args) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_sizes(torch_cuda):
    torch = torch_cuda
    from paper_1309_3075_b300.binding import epoch_site_log_sum_noalloc
    dev = torch.device("cuda", 0)
    a = torch.zeros(64, dtype=torch.float64, device=dev)
    ex = torch.zeros(64, dtype=torch.int16, device=dev)
    ptr = a.data_ptr()
    # too many patterns: EPOCH_ERR_CAPACITY, nothing launched
    assert epoch_site_log_sum_noalloc(ptr, 0, 0, 0, ptr, MAX_PATTERNS + 1, 0, ptr) == 3
    # row stride shorter than a row, negative size, missing output: EPOCH_ERR_ARG
    assert epoch_site_log_sum_noalloc(ptr, ex.data_ptr(), 1, 10, ptr, 20, 0, ptr) == 1
    assert epoch_site_log_sum_noalloc(ptr, 0, 0, 0, ptr, -1, 0, ptr) == 1
    assert epoch_site_log_sum_noalloc(ptr, 0, 0, 0, ptr, 10, 0, 0) == 1
    # no patterns: lnL = 0
    a[0] = 5.0
    assert epoch_site_log_sum_noalloc(0, 0, 0, 0, 0, 0, 0, ptr) == 0
    torch.cuda.synchronize()
    assert float(a[0].item()) == 0.0
