// k_stage.cu -- the per-step host <-> device transfers of a context as
// kernels on its stream.
//
// An inference step moves a few kilobytes each way: the parameters that
// changed (Q, pi, dQ, boundaries, categories, heights) in, and the lnL, the
// status word and the gradient out.  At that size a copy-engine transfer is
// all latency: the copy is queued on another engine and the next kernel waits
// on its completion semaphore.  These kernels instead read the pinned host
// mirror (mapped into the device's address space) and write the pinned result
// mirror directly, in stream order with the evaluation, so nothing crosses
// engines.  Each thread moves one double per pass; one pass covers up to
// 148 x 256 doubles.
#include <cuda_runtime.h>

#include "epoch_internal.cuh"

namespace epoch {
namespace {

struct StageSeg {
  const double *src;
  double *dst;
  size_t n;
};

struct StageArgs {
  StageSeg seg[2];
};

// blockIdx.y selects the segment
__global__ void __launch_bounds__(256) k_stage(StageArgs a) {
  const StageSeg s = a.seg[blockIdx.y];
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += stride)
    s.dst[i] = s.src[i];
}

}  // namespace

// Copies n0 doubles src0 -> dst0 and n1 doubles src1 -> dst1 (n1 may be 0)
// on the stream; either side may be device memory or mapped pinned host
// memory (its device address).
cudaError_t launch_stage(const double *src0, double *dst0, size_t n0, const double *src1,
                         double *dst1, size_t n1, cudaStream_t stream) {
  StageArgs a;
  a.seg[0] = {src0, dst0, n0};
  a.seg[1] = {src1, dst1, n1};
  const size_t n = n0 > n1 ? n0 : n1;
  if (n == 0) return cudaSuccess;
  size_t blocks = (n + 255) / 256;
  if (blocks > 148) blocks = 148;
  k_stage<<<dim3((unsigned)blocks, n1 > 0 ? 2u : 1u), 256, 0, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace epoch
