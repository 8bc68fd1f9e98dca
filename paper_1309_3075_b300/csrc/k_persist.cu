// k_persist.cu -- single-launch, dependency-driven post-order and pre-order
// passes for the FP32 K = 4 path.
//
// Site patterns are independent (paper, Methods: sites and rate categories
// are conditionally independent and their contributions aggregate), so the
// unit of work is (internal node u, tile of kPTile patterns).  Items are
// handed out by an atomic counter in post-order level order (pre-order:
// reverse order); an item waits only for the items of the same tile at its
// children (pre-order: its parent), which were handed out earlier to CTAs
// that are running, so the smallest unfinished item can always proceed.
// Every wait is bounded: on expiry the kernel sets ST_TIMEOUT, raises an
// abort word that makes the other CTAs stop waiting, and finishes.
//
// Producer: all threads store, __syncthreads, thread 0 fences and
// release-stores the tile's flag.  Consumer: thread 0 acquire-loads the
// flag, __syncthreads, all threads load through L2 (ld.global.cg) so no
// stale L1 line from an earlier evaluation is used.
#include <math.h>

#include <algorithm>

#include "epoch_internal.cuh"

namespace epoch {
namespace {

constexpr int kThreads = 256;
constexpr int kPTile = 512;          // patterns per work item (2 per thread)
constexpr int kSpinLimit = 1 << 21;  // ~2 s of polling at ~1 us per poll

__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int *p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bounded wait for *flag != 0 by one thread.  ctl[3] is the abort word.
__device__ void wait_flag(const int *flag, int *ctl, int *status) {
  int spins = 0;
  while (ld_acquire(flag) == 0) {
    if (ld_acquire(ctl + 3) != 0) return;
    if (++spins > kSpinLimit) {
      atomicOr(status, ST_TIMEOUT);
      atomicExch(ctl + 3, 1);
      return;
    }
    __nanosleep(256);
  }
}

__device__ __forceinline__ float4 matvec_t(const float4 *t, float4 l) {
  float4 s;
  s.x = l.x * t[0].x + l.y * t[1].x + l.z * t[2].x + l.w * t[3].x;
  s.y = l.x * t[0].y + l.y * t[1].y + l.z * t[2].y + l.w * t[3].y;
  s.z = l.x * t[0].z + l.y * t[1].z + l.z * t[2].z + l.w * t[3].z;
  s.w = l.x * t[0].w + l.y * t[1].w + l.z * t[2].w + l.w * t[3].w;
  return s;
}
__device__ __forceinline__ float4 mul4(float4 a, float4 b) {
  return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w);
}
__device__ __forceinline__ float dot4(float4 a, float4 b) {
  return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
}
__device__ __forceinline__ float4 ldexp4(float4 a, int e) {
  return make_float4(ldexpf(a.x, -e), ldexpf(a.y, -e), ldexpf(a.z, -e), ldexpf(a.w, -e));
}

__device__ __forceinline__ float reduce_scatter32(float (&v)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 16; k++) {
    const bool up = lane & 16;
    const float send = up ? v[k] : v[k + 16];
    const float keep = up ? v[k + 16] : v[k];
    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int k = 0; k < 8; k++) {
    const bool up = lane & 8;
    const float send = up ? v[k] : v[k + 8];
    const float keep = up ? v[k + 8] : v[k];
    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const bool up = lane & 4;
    const float send = up ? v[k] : v[k + 4];
    const float keep = up ? v[k + 4] : v[k];
    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
#pragma unroll
  for (int k = 0; k < 2; k++) {
    const bool up = lane & 2;
    const float send = up ? v[k] : v[k + 2];
    const float keep = up ? v[k + 2] : v[k];
    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  {
    const bool up = lane & 1;
    const float send = up ? v[0] : v[1];
    const float keep = up ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 1);
  }
  return v[0];
}

struct PassArgs {
  Dims d;
  const float *PT32;
  const int *nodes;   // internal nodes in post-order level order
  int n_int;          // N-1
  int ntile;
  const int *child;
  float4 *part;
  float4 *pre;
  int16_t *scale;
  const uint8_t *tips;
  const unsigned long long *masks;
  const double *pi;
  const double *catw;
  const double *pw;
  int root;
  int *flags;         // [N-1][ntile]
  int *ctl;           // [0] queue, [3] abort
  double *site_log;   // [P] log of the scaled root sum
  double *site_inv;   // [P] 1 / scaled root sum
  float *Gpart;       // [N-1][ntile][2][C][16]
  int *status;
};

// ---- post-order: pruning + rescaling (+ root sums on the root's items) ----
template <int CMAX>
__global__ void __launch_bounds__(kThreads) k_post_k4(PassArgs a) {
  extern __shared__ float4 spt[];  // [2][C][NR]
  __shared__ int s_item;
  const Dims &d = a.d;
  const int CN = d.C * d.NR;
  const int n_items = a.n_int * a.ntile;
  const float4 *pt4 = reinterpret_cast<const float4 *>(a.PT32);
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(a.ctl, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= n_items) break;
    const int ni = item / a.ntile, t = item - ni * a.ntile;
    const int u = a.nodes[ni], slot = u - d.N;
    const int ch0 = a.child[2 * slot], ch1 = a.child[2 * slot + 1];
    if (threadIdx.x == 0) {
      if (ch0 >= d.N) wait_flag(a.flags + (size_t)(ch0 - d.N) * a.ntile + t, a.ctl, a.status);
      if (ch1 >= d.N) wait_flag(a.flags + (size_t)(ch1 - d.N) * a.ntile + t, a.ctl, a.status);
    }
    for (int idx = threadIdx.x; idx < 2 * CN; idx += blockDim.x) {
      const int x = idx / CN, r = idx - x * CN;
      spt[idx] = pt4[(size_t)(x ? ch1 : ch0) * CN + r];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kPTile / kThreads; k++) {
      const int p = t * kPTile + k * kThreads + threadIdx.x;
      if (p >= d.P) continue;
      float4 acc[CMAX];
#pragma unroll
      for (int c = 0; c < CMAX; c++) acc[c] = make_float4(1.f, 1.f, 1.f, 1.f);
#pragma unroll
      for (int x = 0; x < 2; x++) {
        const int node = x ? ch1 : ch0;
        const float4 *tab = spt + x * CN;
        if (node < d.N) {
          const int code = a.tips[(size_t)node * d.P + p];
#pragma unroll
          for (int c = 0; c < CMAX; c++)
            if (c < d.C) acc[c] = mul4(acc[c], tab[c * d.NR + code]);
        } else {
          const float4 *L = a.part + (size_t)(node - d.N) * d.C * d.P + p;
          float4 l[CMAX];
#pragma unroll
          for (int c = 0; c < CMAX; c++)
            if (c < d.C) l[c] = __ldcg(L + (size_t)c * d.P);
#pragma unroll
          for (int c = 0; c < CMAX; c++)
            if (c < d.C) acc[c] = mul4(acc[c], matvec_t(tab + c * d.NR, l[c]));
        }
      }
      float m = 0.f;
#pragma unroll
      for (int c = 0; c < CMAX; c++)
        if (c < d.C) m = fmaxf(m, fmaxf(fmaxf(acc[c].x, acc[c].y), fmaxf(acc[c].z, acc[c].w)));
      int e = 0;
      if (!isfinite(m)) {
        atomicOr(a.status, ST_NONFINITE);
      } else if (m > 0.f) {
        frexpf(m, &e);
      }
      float4 *out = a.part + (size_t)slot * d.C * d.P + p;
      double site = 0.0;
#pragma unroll
      for (int c = 0; c < CMAX; c++) {
        if (c < d.C) {
          const float4 v = ldexp4(acc[c], e);
          out[(size_t)c * d.P] = v;
          if (u == a.root)
            site += a.catw[c] * (a.pi[0] * v.x + a.pi[1] * v.y + a.pi[2] * v.z + a.pi[3] * v.w);
        }
      }
      a.scale[(size_t)slot * d.P + p] = (int16_t)e;
      if (u == a.root) {
        a.site_log[p] = log(site);
        a.site_inv[p] = site > 0.0 ? 1.0 / site : 0.0;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      st_release(a.flags + (size_t)slot * a.ntile + t, 1);
    }
  }
}

// ---- pre-order: outside partials and per-tile sums of G ------------------
template <int CMAX>
__global__ void __launch_bounds__(kThreads) k_pre_k4p(PassArgs a) {
  extern __shared__ float4 spt[];  // [2][C][NR] tables, then [nwarp][C][32] sums
  __shared__ int s_item;
  const Dims &d = a.d;
  const int CN = d.C * d.NR;
  const int n_items = a.n_int * a.ntile;
  const float4 *pt4 = reinterpret_cast<const float4 *>(a.PT32);
  float *wsum = reinterpret_cast<float *>(spt + 2 * CN);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int nw = kThreads / 32;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(a.ctl, 1);
    __syncthreads();
    const int j = s_item;
    if (j >= n_items) break;
    const int ni = a.n_int - 1 - j / a.ntile, t = j % a.ntile;
    const int u = a.nodes[ni], slot = u - d.N;
    const int ch0 = a.child[2 * slot], ch1 = a.child[2 * slot + 1];
    const bool is_root = (u == a.root);
    if (threadIdx.x == 0 && !is_root)
      wait_flag(a.flags + (size_t)slot * a.ntile + t, a.ctl, a.status);
    for (int idx = threadIdx.x; idx < 2 * CN; idx += blockDim.x) {
      const int x = idx / CN, r = idx - x * CN;
      spt[idx] = pt4[(size_t)(x ? ch1 : ch0) * CN + r];
    }
    __syncthreads();
    for (int c = 0; c < d.C; c++) {
      const float4 *t0 = spt + c * d.NR, *t1 = spt + CN + c * d.NR;
      float g[32];
#pragma unroll
      for (int q = 0; q < 32; q++) g[q] = 0.f;
#pragma unroll
      for (int k = 0; k < kPTile / kThreads; k++) {
        const int p = t * kPTile + k * kThreads + threadIdx.x;
        if (p >= d.P) continue;
        const int e = a.scale[(size_t)slot * d.P + p];
        const float n = (float)a.pw[p];
        float4 uu;
        if (is_root) {
          const float wc = (float)(a.catw[c] * a.site_inv[p]);
          uu = make_float4(wc * (float)a.pi[0], wc * (float)a.pi[1], wc * (float)a.pi[2],
                           wc * (float)a.pi[3]);
        } else {
          uu = __ldcg(a.pre + ((size_t)slot * d.C + c) * d.P + p);
        }
        float4 l0, l1, s0, s1;
        if (ch0 < d.N) {
          const int code = a.tips[(size_t)ch0 * d.P + p];
          s0 = t0[code];
          const unsigned long long mk =
              code < 4 ? (1ull << code) : (code == 4 ? ~0ull : a.masks[code - 5]);
          l0 = make_float4((mk & 1ull) ? 1.f : 0.f, (mk & 2ull) ? 1.f : 0.f,
                           (mk & 4ull) ? 1.f : 0.f, (mk & 8ull) ? 1.f : 0.f);
        } else {
          l0 = __ldcs(a.part + ((size_t)(ch0 - d.N) * d.C + c) * d.P + p);
          s0 = matvec_t(t0, l0);
        }
        if (ch1 < d.N) {
          const int code = a.tips[(size_t)ch1 * d.P + p];
          s1 = t1[code];
          const unsigned long long mk =
              code < 4 ? (1ull << code) : (code == 4 ? ~0ull : a.masks[code - 5]);
          l1 = make_float4((mk & 1ull) ? 1.f : 0.f, (mk & 2ull) ? 1.f : 0.f,
                           (mk & 4ull) ? 1.f : 0.f, (mk & 8ull) ? 1.f : 0.f);
        } else {
          l1 = __ldcs(a.part + ((size_t)(ch1 - d.N) * d.C + c) * d.P + p);
          s1 = matvec_t(t1, l1);
        }
        const float4 x0 = ldexp4(mul4(uu, s1), e);
        const float4 x1 = ldexp4(mul4(uu, s0), e);
        if (ch0 >= d.N)
          a.pre[((size_t)(ch0 - d.N) * d.C + c) * d.P + p] =
              make_float4(dot4(t0[0], x0), dot4(t0[1], x0), dot4(t0[2], x0), dot4(t0[3], x0));
        if (ch1 >= d.N)
          a.pre[((size_t)(ch1 - d.N) * d.C + c) * d.P + p] =
              make_float4(dot4(t1[0], x1), dot4(t1[1], x1), dot4(t1[2], x1), dot4(t1[3], x1));
        const float xa[4] = {x0.x * n, x0.y * n, x0.z * n, x0.w * n};
        const float la[4] = {l0.x, l0.y, l0.z, l0.w};
        const float xb[4] = {x1.x * n, x1.y * n, x1.z * n, x1.w * n};
        const float lb[4] = {l1.x, l1.y, l1.z, l1.w};
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
          for (int jj = 0; jj < 4; jj++) {
            g[i * 4 + jj] += xa[i] * la[jj];
            g[16 + i * 4 + jj] += xb[i] * lb[jj];
          }
      }
      wsum[(warp * d.C + c) * 32 + lane] = reduce_scatter32(g);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < d.C * 32; q += blockDim.x) {
      const int c = q >> 5, l = q & 31;
      float s = 0.f;
      for (int w = 0; w < nw; w++) s += wsum[(w * d.C + c) * 32 + l];
      const int xch = l >> 4, ij = l & 15;
      a.Gpart[((((size_t)slot * a.ntile + t) * 2 + xch) * d.C + c) * 16 + ij] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      if (ch0 >= d.N) st_release(a.flags + (size_t)(ch0 - d.N) * a.ntile + t, 1);
      if (ch1 >= d.N) st_release(a.flags + (size_t)(ch1 - d.N) * a.ntile + t, 1);
    }
  }
}

// ---- per-pattern log-likelihood and the weighted log-sum -----------------
// lnL_p = log(scaled root sum) + ln2 * sum_u e_u(p); the exponent sum is
// split over 8 node groups per pattern.  Block partial sums of n_p lnL_p are
// reduced in a fixed order by the last block to finish (deterministic).
__global__ void __launch_bounds__(256) k_site_lnl(Dims d, const int16_t *__restrict__ scale,
                                                  const double *__restrict__ site_log,
                                                  const double *__restrict__ pw,
                                                  double *__restrict__ site_lnl,
                                                  double *__restrict__ part, int *ctl,
                                                  double *__restrict__ lnl) {
  __shared__ int es[8][32];
  __shared__ double red[8];
  __shared__ int s_last;
  const int pl = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int p = blockIdx.x * 32 + pl;
  int acc = 0;
  if (p < d.P)
    for (int s = g; s < d.N - 1; s += 8) acc += scale[(size_t)s * d.P + p];
  es[g][pl] = acc;
  __syncthreads();
  double contrib = 0.0;
  if (g == 0 && p < d.P) {
    int tot = 0;
    for (int k = 0; k < 8; k++) tot += es[k][pl];
    const double lp = site_log[p] + 0.69314718055994530942 * (double)tot;
    site_lnl[p] = lp;
    const double n = pw[p];
    contrib = (n != 0.0) ? n * lp : 0.0;
  }
  if (g == 0) {
    for (int o = 16; o > 0; o >>= 1) contrib += __shfl_xor_sync(0xffffffffu, contrib, o);
    if (pl == 0) {
      part[blockIdx.x] = contrib;
      __threadfence();
      s_last = (atomicAdd(ctl + 4, 1) == (int)gridDim.x - 1);
    }
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double t = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += __ldcg(part + i);
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (pl == 0) red[g] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < 8; k++) s += red[k];
    lnl[0] = s;
  }
}

template <typename K>
int grid_for(K kernel, size_t smem) {
  int dev = 0, sms = 148, per = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kThreads, smem);
  return sms * (per > 0 ? per : 1);
}

PassArgs make_args(epoch_ctx *c, int root) {
  PassArgs a;
  a.d = c->d;
  a.PT32 = c->d_PT32;
  a.nodes = c->d_level_nodes;
  a.n_int = c->d.N - 1;
  a.ntile = ceil_div(c->d.P, kPTile);
  a.child = c->d_child;
  a.part = reinterpret_cast<float4 *>(c->d_part);
  a.pre = reinterpret_cast<float4 *>(c->d_pre);
  a.scale = c->d_scale;
  a.tips = c->d_tips;
  a.masks = c->d_masks;
  a.pi = c->d_pi;
  a.catw = c->d_catw;
  a.pw = c->d_pw;
  a.root = root;
  a.flags = c->d_flags;
  a.ctl = c->d_ctl;
  a.site_log = c->d_site_log;
  a.site_inv = c->d_site_inv;
  a.Gpart = (float *)c->d_Gpart;
  a.status = c->d_status;
  return a;
}

int root_of(const epoch_ctx *c) {
  for (int v = 0; v < c->d.nn; v++)
    if (c->h_parent[v] < 0) return v;
  return -1;
}

template <int CMAX>
cudaError_t post_k4(epoch_ctx *c) {
  PassArgs a = make_args(c, root_of(c));
  const size_t smem = sizeof(float4) * 2 * c->d.C * c->d.NR;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_post_k4<CMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const size_t nflag = (size_t)a.n_int * a.ntile;
  cudaMemsetAsync(c->d_flags, 0, nflag * sizeof(int), c->stream);
  cudaMemsetAsync(c->d_ctl, 0, 8 * sizeof(int), c->stream);
  const int grid = std::min(grid_for(k_post_k4<CMAX>, smem), (int)nflag);
  k_post_k4<CMAX><<<grid, kThreads, smem, c->stream>>>(a);
  const int nb = ceil_div(c->d.P, 32);
  k_site_lnl<<<nb, 256, 0, c->stream>>>(c->d, c->d_scale, c->d_site_log, c->d_pw, c->d_site_lnl,
                                         c->d_lnl_part, c->d_ctl, c->d_lnl);
  c->launches += 2;
  return cudaGetLastError();
}

template <int CMAX>
cudaError_t pre_k4(epoch_ctx *c) {
  PassArgs a = make_args(c, root_of(c));
  const size_t smem =
      sizeof(float4) * 2 * c->d.C * c->d.NR + sizeof(float) * (kThreads / 32) * c->d.C * 32;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_pre_k4p<CMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const size_t nflag = (size_t)a.n_int * a.ntile;
  cudaMemsetAsync(c->d_flags, 0, nflag * sizeof(int), c->stream);
  cudaMemsetAsync(c->d_ctl, 0, 8 * sizeof(int), c->stream);
  const int grid = std::min(grid_for(k_pre_k4p<CMAX>, smem), (int)nflag);
  k_pre_k4p<CMAX><<<grid, kThreads, smem, c->stream>>>(a);
  c->launches++;
  return cudaGetLastError();
}

}  // namespace

int persist_tile() { return kPTile; }

cudaError_t launch_partials_k4(epoch_ctx *c) {
  if (c->d.C <= 4) return post_k4<4>(c);
  if (c->d.C <= 8) return post_k4<8>(c);
  return post_k4<16>(c);
}

cudaError_t launch_preorder_k4(epoch_ctx *c) {
  if (c->d.C <= 4) return pre_k4<4>(c);
  if (c->d.C <= 8) return pre_k4<8>(c);
  return pre_k4<16>(c);
}

}  // namespace epoch
