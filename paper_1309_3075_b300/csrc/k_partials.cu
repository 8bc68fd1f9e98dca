// k_partials.cu -- post-order pruning (Eq. partial_likelihood) with
// per-pattern power-of-two rescaling, and the root sum / weighted log-sum.
//
// Layout: partials of internal node u live at slot u-N as [C][P][Kp]; a
// pattern's state vector is contiguous (Kp = 4 for K <= 4: one 16-byte
// vector).  Tips are never expanded: a tip child contributes the row of the
// transposed branch-matrix table selected by its code (FP32 paths) or the
// column / masked row-sum of P (FP64 path).  After each internal node the
// pattern's values over (category, state) are divided by 2^e, e the binary
// exponent of their maximum, which is exact; e is kept per (node, pattern).
#include <math.h>

#include "branch_table.cuh"

namespace epoch {
namespace {

// ---- generic kernels (any K; FP64 = the plain path, FP32 = SIMT path) -----

// One thread per (category, pattern, state) of one node of the level.
template <typename T>
__global__ void k_partials_generic(Dims d, BranchTable<T> bt, const int *__restrict__ lvl_nodes,
                                   int lvl_off, const int *__restrict__ child, T *part,
                                   const uint8_t *__restrict__ tips) {
  const int u = lvl_nodes[lvl_off + blockIdx.y];
  const int slot = u - d.N;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)d.C * d.P * d.Kp) return;
  const int i = (int)(idx % d.Kp);
  const long long cp = idx / d.Kp;
  const int p = (int)(cp % d.P), c = (int)(cp / d.P);
  T out = 0;
  if (i < d.K) {
    const int v = child[2 * slot], w = child[2 * slot + 1];
    out = child_factor<T>(d, bt, part, tips, v, c, p, i) *
          child_factor<T>(d, bt, part, tips, w, c, p, i);
  }
  part[(((size_t)slot * d.C + c) * d.P + p) * d.Kp + i] = out;
}

// One thread per (node of the level, pattern): divide by 2^e of the max.
template <typename T>
__global__ void k_rescale_generic(Dims d, const int *__restrict__ lvl_nodes, int lvl_off, T *part,
                                  int16_t *__restrict__ scale, int *__restrict__ status) {
  const int u = lvl_nodes[lvl_off + blockIdx.y];
  const int slot = u - d.N;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= d.P) return;
  T m = 0;
  for (int c = 0; c < d.C; c++) {
    const T *L = part + (((size_t)slot * d.C + c) * d.P + p) * d.Kp;
    for (int i = 0; i < d.K; i++) m = fmax(m, L[i]);
  }
  int e = 0;
  if (!isfinite(m)) {
    atomicOr(status, ST_NONFINITE);
  } else if (m > 0) {
    e = exp_of(m);
    for (int c = 0; c < d.C; c++) {
      T *L = part + (((size_t)slot * d.C + c) * d.P + p) * d.Kp;
      for (int i = 0; i < d.K; i++) L[i] = scale_by(L[i], e);
    }
  }
  scale[(size_t)slot * d.Pp + p] = (int16_t)e;
}

// ---- root: per-pattern site likelihood and the weighted log-sum ----------
// site_p = sum_c w_c sum_i pi_i L_root(c,p,i) (scaled), lnL_p = log site_p +
// ln2 * sum_u e_u(p); the block sums of n_p lnL_p are reduced in a fixed
// order by k_lnl_final (deterministic).
template <typename T>
__global__ void k_root(Dims d, int root_slot, const T *__restrict__ part,
                       const int16_t *__restrict__ scale, const double *__restrict__ pi,
                       const double *__restrict__ catw, const double *__restrict__ pw,
                       double *__restrict__ site_lnl, double *__restrict__ site_inv,
                       double *__restrict__ lnl_part) {
  __shared__ double red[32];
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  double contrib = 0.0;
  if (p < d.P) {
    double site = 0.0;
    for (int c = 0; c < d.C; c++) {
      const T *L = part + (((size_t)root_slot * d.C + c) * d.P + p) * d.Kp;
      double sc = 0.0;
      for (int i = 0; i < d.K; i++) sc += pi[i] * (double)L[i];
      site += catw[c] * sc;
    }
    int esum = 0;
    for (int s = 0; s < d.N - 1; s++) esum += scale[(size_t)s * d.Pp + p];
    const double lp = log(site) + 0.69314718055994530942 * (double)esum;
    site_lnl[p] = lp;
    site_inv[p] = site > 0.0 ? 1.0 / site : 0.0;
    const double n = pw[p];
    contrib = (n != 0.0) ? n * lp : 0.0;
  }
  for (int o = 16; o > 0; o >>= 1) contrib += __shfl_xor_sync(0xffffffffu, contrib, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = contrib;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += red[i];
    lnl_part[blockIdx.x] = t;
  }
}

__global__ void k_lnl_final(int n, const double *__restrict__ part, double *__restrict__ out) {
  __shared__ double red[32];
  double t = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) t += part[i];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) s += red[i];
    out[0] = s;
  }
}

template <typename T>
cudaError_t launch_generic_levels(epoch_ctx *c, BranchTable<T> bt) {
  const Dims &d = c->d;
  const int L = (int)c->h_level_off.size() - 1;
  const long long items = (long long)d.C * d.P * d.Kp;
  for (int l = 0; l < L; l++) {
    const int w = c->h_level_off[l + 1] - c->h_level_off[l];
    if (sizeof(T) == sizeof(float) && tc_path(c)) {  // tile products on the tensor cores
      cudaError_t e = launch_tc_post(c, l);
      if (e != cudaSuccess) return e;
      continue;
    }
    dim3 g1(ceil_div(items, 256), w);
    k_partials_generic<T><<<g1, 256, 0, c->stream>>>(d, bt, c->d_level_nodes, c->h_level_off[l],
                                                     c->d_child, (T *)c->d_part, c->d_tips);
    dim3 g2(ceil_div(d.P, 256), w);
    k_rescale_generic<T><<<g2, 256, 0, c->stream>>>(d, c->d_level_nodes, c->h_level_off[l],
                                                    (T *)c->d_part, c->d_scale, c->d_status);
    c->launches += 2;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_partials(epoch_ctx *c) {
  const Dims &d = c->d;
  if (small_path(c)) return launch_small_post(c);  // includes the root log-sum
  if (c->precision == EPOCH_FP64) {
    BranchTable<double> bt{c->d_P64, c->d_masks};
    return launch_generic_levels<double>(c, bt);
  }
  if (fast_k4(c)) return launch_partials_k4(c);  // includes the root log-sum
  BranchTable<float> bt{c->d_PT32, c->d_masks};
  return launch_generic_levels<float>(c, bt);
}

cudaError_t launch_root(epoch_ctx *c) {
  const Dims &d = c->d;
  if (fast_k4(c) || small_path(c)) return cudaSuccess;  // done by the pruning pass
  int root_slot = -1;
  for (int v = 0; v < d.nn; v++)
    if (c->h_parent[v] < 0) root_slot = v - d.N;
  const int nb = ceil_div(d.P, kTile);
  if (c->precision == EPOCH_FP64)
    k_root<double><<<nb, kTile, 0, c->stream>>>(d, root_slot, (const double *)c->d_part,
                                                c->d_scale, c->d_pi, c->d_catw, c->d_pw,
                                                c->d_site_lnl, c->d_site_inv, c->d_lnl_part);
  else
    k_root<float><<<nb, kTile, 0, c->stream>>>(d, root_slot, (const float *)c->d_part,
                                               c->d_scale, c->d_pi, c->d_catw, c->d_pw,
                                               c->d_site_lnl, c->d_site_inv, c->d_lnl_part);
  k_lnl_final<<<1, 256, 0, c->stream>>>(nb, c->d_lnl_part, c->d_lnl);
  c->launches += 2;
  return cudaGetLastError();
}

}  // namespace epoch
