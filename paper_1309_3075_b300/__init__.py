"""B300 (sm_103a) library for the tree likelihood and its gradient under the
epoch (time-heterogeneous) substitution model of Bielejec et al.
(arXiv 1309.3075).

The compute path is libepoch.so (CUDA kernels behind the C ABI of
include/epoch.h); ``binding`` marshals arguments to it and ``autograd`` wraps
it in a torch.autograd.Function.  Build with ``python -m
paper_1309_3075_b300.build``.
"""
from paper_1309_3075_b300.binding import (  # noqa: F401
    EPOCH_FP32,
    EPOCH_FP32_TC,
    EPOCH_FP64,
    EpochError,
    EpochLikelihood,
    lib,
)
