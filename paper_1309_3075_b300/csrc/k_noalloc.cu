// k_noalloc.cu -- epoch_site_log_sum_noalloc: the per-pattern log-sum of the
// root step with every byte of scratch in one static device array, so the
// call itself never allocates device memory.
//
// Who needs this: a caller whose device memory is fixed up front cannot let a
// library allocate behind its back -- an MCMC or optimiser loop that must run
// for days at a constant footprint, a host program that has already handed
// almost all HBM to its own pool (a framework's caching allocator), or code
// that wants the same addresses on every call.  The context-based entry
// points keep their block sums and counters in buffers made by
// epoch_create; this one keeps them in noalloc_scratch below.
//
// What it computes is the last step of the root (Methods, the log-likelihood
// as a weighted sum over patterns):
//   site_out[p] = site_log[p] + ln 2 * sum_{u < rows} exponents[u][p]
//   lnL         = sum_p w_p site_out[p]     (terms with w_p = 0 skipped)
// with the block sums reduced in a fixed order by the last block to finish,
// so the result does not depend on scheduling.
//
// Scratch rules:
//   * noalloc_scratch holds kNoallocMaxBlocks block sums followed by the
//     block counter.  The counter must be zero when a launch starts: the
//     first call on a device zeroes it (cudaMemsetAsync on the caller's
//     stream), and every launch's last block sets it back to zero.
//   * The first call on each device also looks up the array's device address
//     with cudaGetSymbolAddress (with that device current) and keeps it; make
//     that first call before any stream capture begins.
//   * There is one scratch array per device: two calls on the same device
//     that can overlap in time (different streams, different host threads)
//     race on it.  Callers must order such calls.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "epoch.h"

namespace {

constexpr int kPatternsPerBlock = 32;
constexpr int kNoallocMaxBlocks = EPOCH_NOALLOC_MAX_PATTERNS / kPatternsPerBlock;
constexpr int kMaxDevices = 64;

// [kNoallocMaxBlocks] block sums, then the counter (as unsigned int) in the
// first word of the 32 slots after them.
static __device__ __align__(256) double noalloc_scratch[kNoallocMaxBlocks + 32];

__global__ void __launch_bounds__(256) k_site_log_sum_noalloc(
    const double *__restrict__ site_log, const int16_t *__restrict__ ex, int rows, long long stride,
    const double *__restrict__ w, int P, double *__restrict__ site_out, double *__restrict__ lnl,
    double *scratch) {
  __shared__ int es[8][32];
  __shared__ double redd[8];
  __shared__ int s_last;
  unsigned int *counter = reinterpret_cast<unsigned int *>(scratch + kNoallocMaxBlocks);
  const int pl = threadIdx.x & 31, gi = threadIdx.x >> 5;
  const int p = blockIdx.x * kPatternsPerBlock + pl;
  int acc = 0;
  if (p < P)
    for (int s = gi; s < rows; s += 8) acc += ex[(size_t)s * stride + p];
  es[gi][pl] = acc;
  __syncthreads();
  double contrib = 0.0;
  if (gi == 0 && p < P) {
    int tot = 0;
    for (int k = 0; k < 8; k++) tot += es[k][pl];
    const double lp = site_log[p] + 0.69314718055994530942 * (double)tot;
    if (site_out) site_out[p] = lp;
    const double nw = w[p];
    contrib = (nw != 0.0) ? nw * lp : 0.0;
  }
  if (gi == 0) {
    for (int o = 16; o > 0; o >>= 1) contrib += __shfl_xor_sync(0xffffffffu, contrib, o);
    if (pl == 0) {
      scratch[blockIdx.x] = contrib;
      __threadfence();
      s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double t = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += __ldcg(scratch + i);
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (pl == 0) redd[gi] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < 8; k++) s += redd[k];
    lnl[0] = s;
    *counter = 0u;  // ready for the next launch
  }
}

std::mutex g_setup_mutex;
double *g_scratch[kMaxDevices] = {};

}  // namespace

extern "C" epoch_status epoch_site_log_sum_noalloc(const double *site_log,
                                                   const int16_t *exponents, int n_rows,
                                                   long long row_stride, const double *weights,
                                                   int n_patterns, double *site_out,
                                                   double *lnL_out, void *cuda_stream) {
  if (n_patterns < 0 || n_rows < 0 || !lnL_out) return EPOCH_ERR_ARG;
  if (n_patterns > 0 && (!site_log || !weights)) return EPOCH_ERR_ARG;
  if (n_rows > 0 && n_patterns > 0 && (!exponents || row_stride < n_patterns))
    return EPOCH_ERR_ARG;
  if (n_patterns > EPOCH_NOALLOC_MAX_PATTERNS) return EPOCH_ERR_CAPACITY;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return EPOCH_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return EPOCH_ERR_CAPACITY;
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  double *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch[dev]) {
      void *ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, noalloc_scratch) != cudaSuccess || !ptr)
        return EPOCH_ERR_CUDA;
      double *base = static_cast<double *>(ptr);
      if (cudaMemsetAsync(base + kNoallocMaxBlocks, 0, sizeof(unsigned int), stream) !=
          cudaSuccess)
        return EPOCH_ERR_CUDA;
      g_scratch[dev] = base;
    }
    scratch = g_scratch[dev];
  }
  const int blocks = n_patterns > 0 ? (n_patterns + kPatternsPerBlock - 1) / kPatternsPerBlock : 1;
  k_site_log_sum_noalloc<<<blocks, 256, 0, stream>>>(site_log, n_rows > 0 ? exponents : nullptr,
                                                     n_patterns > 0 ? n_rows : 0, row_stride,
                                                     weights, n_patterns, site_out, lnL_out,
                                                     scratch);
  return cudaGetLastError() == cudaSuccess ? EPOCH_OK : EPOCH_ERR_CUDA;
}
