"""torch.autograd.Function over the library: gradients from backward() against
the FP64 oracle's gradient, with heights as CUDA tensors (device pointers in
and out, no host round trip) and as host tensors."""
import numpy as np
import pytest

import oracle
import synth
from tolerances import grad_close

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec_name", ["fp64", "fp32"])
@pytest.mark.parametrize("device_heights", [True, False])
def test_backward_matches_oracle_gradient(prec_name, device_heights):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1309_3075_b300.autograd import log_likelihood
    from paper_1309_3075_b300.binding import EPOCH_FP32, EPOCH_FP64, EpochLikelihood

    prec = EPOCH_FP64 if prec_name == "fp64" else EPOCH_FP32
    w = synth.small_nucleotide(606, n_taxa=12, n_sites=200, n_cat=2, n_epochs=3, dated=True)
    ref = oracle.gradient(w)
    stream = torch.cuda.Stream()  # a stream torch and the library both name
    lik = EpochLikelihood(w, precision=prec, cuda_stream=stream.cuda_stream)
    try:
        dQ = np.asarray(w.dQ)

        def model_fn(th):  # Q(theta) = Q + sum_a theta_a dQ_a, so theta = 0 gives w.Q
            return np.asarray(w.Q) + np.tensordot(th, dQ, axes=1), dQ

        dev = torch.device("cuda", 0) if device_heights else torch.device("cpu")
        heights = torch.tensor(w.heights, dtype=torch.float64, device=dev, requires_grad=True)
        bounds = torch.tensor(w.boundaries, dtype=torch.float64, requires_grad=True)
        theta = torch.zeros(dQ.shape[0], dtype=torch.float64, requires_grad=True)
        with torch.cuda.stream(stream):
            lnl = log_likelihood(lik, model_fn, w.pi, heights, bounds, theta)
            assert lnl.device.type == ("cuda" if device_heights else "cpu")
            lnl.backward()
        torch.cuda.synchronize()
        assert abs(float(lnl.detach()) - ref["lnL"]) <= (1e-10 if prec == EPOCH_FP64 else 1e-5) * abs(ref["lnL"])
        assert heights.grad.device == dev
        for got, key in ((heights.grad.cpu().numpy(), "heights"), (bounds.grad.numpy(), "boundaries"),
                         (theta.grad.numpy(), "params")):
            ok, worst = grad_close(got, ref[key], prec)
            assert ok, (key, worst)
    finally:
        lik.close()


def test_device_heights_are_checked_on_the_device():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1309_3075_b300 import binding
    from paper_1309_3075_b300.binding import EPOCH_FP32, EpochError, EpochLikelihood

    w = synth.small_nucleotide(607, n_taxa=8, n_sites=50, n_cat=1, n_epochs=2)
    lik = EpochLikelihood(w, precision=EPOCH_FP32)
    try:
        bad = np.array(w.heights, dtype=np.float64)
        root = int(np.where(np.asarray(w.parent) < 0)[0][0])
        bad[root] = -1.0  # root below its children
        d = torch.tensor(bad, device="cuda")
        torch.cuda.synchronize()
        binding.epoch_set_heights_device(lik.ctx, d.data_ptr())
        binding.epoch_evaluate_async(lik.ctx, 1)
        with pytest.raises(EpochError) as e:
            binding.epoch_read_results(lik.ctx, 2 * w.n_taxa - 1, w.n_epochs, lik.n_params, True)
        assert e.value.status == 1
    finally:
        lik.close()
