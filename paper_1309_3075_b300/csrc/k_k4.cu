// k_k4.cu -- the FP32 path for K = 4 (nucleotides): post-order pruning with
// rescaling, and the pre-order adjoint pass with the per-branch adjoint G,
// organised for HBM bandwidth.
//
//  * One launch per post-order level; grid = (pattern tiles, nodes of the
//    level); a thread owns kPP patterns of one node and keeps every category
//    in registers; the 16-byte state vector of a (category, pattern) is one
//    load.  All loads of a thread are issued before its arithmetic.
//  * Cherries (internal nodes whose two children are tips) are never stored
//    by the post-order pass: L = T_a[code_a] o T_b[code_b] is recomputed from
//    the one-byte tip codes by the parent (two rows of the transposed branch
//    tables; a product of probabilities, so it needs no rescaling, e = 0).
//  * The pre-order pass stores every internal node's outside partial U
//    (cherries included), so each node's step touches exactly its two child
//    branches.  G_{v,c} = sum_p n_p X_v(c,p,:) (x) L_v(c,p,:) is accumulated
//    in registers over the thread's patterns, then reduced over the CTA
//    through shared memory in a fixed order (deterministic) into one tile
//    sum per (branch, tile); k4_G_reduce adds the tile sums in FP64.
#include <math.h>

#include <algorithm>

#include "epoch_internal.cuh"

namespace epoch {
namespace {

constexpr int kThr = 256;          // threads per CTA
constexpr int kPP = 2;             // patterns per thread
constexpr int kK4Tile = kThr * kPP;  // patterns per CTA

__device__ __forceinline__ float4 mul4(float4 a, float4 b) {
  return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w);
}
__device__ __forceinline__ float dot4(float4 a, float4 b) {
  return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
}
__device__ __forceinline__ float4 ldexp4(float4 a, int e) {
  return make_float4(ldexpf(a.x, -e), ldexpf(a.y, -e), ldexpf(a.z, -e), ldexpf(a.w, -e));
}
// S = P L with the transposed table t (t[j] = column j of P): S = sum_j L_j t[j]
__device__ __forceinline__ float4 matvec_t(const float4 *__restrict__ t, float4 l) {
  const float4 r0 = __ldg(t), r1 = __ldg(t + 1), r2 = __ldg(t + 2), r3 = __ldg(t + 3);
  float4 s;
  s.x = l.x * r0.x + l.y * r1.x + l.z * r2.x + l.w * r3.x;
  s.y = l.x * r0.y + l.y * r1.y + l.z * r2.y + l.w * r3.y;
  s.z = l.x * r0.z + l.y * r1.z + l.z * r2.z + l.w * r3.z;
  s.w = l.x * r0.w + l.y * r1.w + l.z * r2.w + l.w * r3.w;
  return s;
}
// U = P^T X: U_j = <t[j], X>
__device__ __forceinline__ float4 matvec(const float4 *__restrict__ t, float4 x) {
  return make_float4(dot4(__ldg(t), x), dot4(__ldg(t + 1), x), dot4(__ldg(t + 2), x),
                     dot4(__ldg(t + 3), x));
}
__device__ __forceinline__ float4 onehot(int code, const unsigned long long *masks) {
  const unsigned long long mk = code < 4 ? (1ull << code) : (code == 4 ? ~0ull : masks[code - 5]);
  return make_float4((mk & 1ull) ? 1.f : 0.f, (mk & 2ull) ? 1.f : 0.f, (mk & 4ull) ? 1.f : 0.f,
                     (mk & 8ull) ? 1.f : 0.f);
}

struct K4Args {
  Dims d;
  const float4 *PT;        // [nn][C][NR] rows of Kp = 4 floats
  const int *nodes;        // internal nodes, level-ascending
  const int *child;        // [N-1][2]
  float4 *part;            // [N-1][C][P]
  float4 *pre;             // [N-1][C][P]
  int16_t *scale;          // [N-1][P]
  const uint8_t *tips;     // [N][P]
  const unsigned long long *masks;
  const double *pi, *catw, *pw;
  int root;
  double *site_log, *site_inv;
  float *Gpart;            // [nn][ntile][C][16] tile sums
  int ntile;
  int *status;
};

// A child of a node: tip, cherry (partial recomputed), or stored.
struct Kid {
  int node, kind, a, b;  // kind 0 tip, 1 cherry, 2 stored; a, b: a cherry's tips
};

__device__ __forceinline__ Kid classify(const K4Args &g, int x) {
  Kid k{x, 0, -1, -1};
  if (x >= g.d.N) {
    const int a = g.child[2 * (x - g.d.N)], b = g.child[2 * (x - g.d.N) + 1];
    if (a < g.d.N && b < g.d.N && x != g.root) {
      k.kind = 1;
      k.a = a;
      k.b = b;
    } else {
      k.kind = 2;
    }
  }
  return k;
}

__device__ __forceinline__ const float4 *tab(const K4Args &g, int node, int c) {
  return g.PT + ((size_t)node * g.d.C + c) * g.d.NR;
}

// Codes a child needs per pattern (tip: its own; cherry: its two tips).
struct KidCodes {
  int c0, c1;
};
__device__ __forceinline__ KidCodes kid_codes(const K4Args &g, const Kid &k, int p) {
  KidCodes r{0, 0};
  if (k.kind == 0) r.c0 = __ldg(g.tips + (size_t)k.node * g.d.P + p);
  if (k.kind == 1) {
    r.c0 = __ldg(g.tips + (size_t)k.a * g.d.P + p);
    r.c1 = __ldg(g.tips + (size_t)k.b * g.d.P + p);
  }
  return r;
}
// L of a child at (c, p): indicator, recomputed cherry partial, or stored.
__device__ __forceinline__ float4 kid_L(const K4Args &g, const Kid &k, const KidCodes &cc, int c,
                                        int p) {
  if (k.kind == 0) return onehot(cc.c0, g.masks);
  if (k.kind == 1) return mul4(__ldg(tab(g, k.a, c) + cc.c0), __ldg(tab(g, k.b, c) + cc.c1));
  // written by an earlier launch, read-only here: the non-coherent path lets
  // these loads move ahead of this thread's stores
  return __ldg(g.part + ((size_t)(k.node - g.d.N) * g.d.C + c) * g.d.P + p);
}
// S = P_x L_x of a child at (c, p).
__device__ __forceinline__ float4 kid_S(const K4Args &g, const Kid &k, const KidCodes &cc, int c,
                                        float4 L) {
  if (k.kind == 0) return __ldg(tab(g, k.node, c) + cc.c0);
  return matvec_t(tab(g, k.node, c), L);
}

// ---- post-order ------------------------------------------------------------
template <int CMAX>
__global__ void __launch_bounds__(kThr, 2) k4_post(K4Args g, int off) {
  const Dims &d = g.d;
  const int u = g.nodes[off + blockIdx.y];
  const int slot = u - d.N;
  const Kid k0 = classify(g, g.child[2 * slot]), k1 = classify(g, g.child[2 * slot + 1]);
  {
    const int p = blockIdx.x * kThr + threadIdx.x;  // one pattern per thread
    if (p >= d.P) return;
    const KidCodes c0 = kid_codes(g, k0, p), c1 = kid_codes(g, k1, p);
    float4 l0[CMAX], l1[CMAX], acc[CMAX];
#pragma unroll
    for (int c = 0; c < CMAX; c++)
      if (c < d.C) {
        l0[c] = k0.kind == 0 ? make_float4(0.f, 0.f, 0.f, 0.f) : kid_L(g, k0, c0, c, p);
        l1[c] = k1.kind == 0 ? make_float4(0.f, 0.f, 0.f, 0.f) : kid_L(g, k1, c1, c, p);
      }
    float m = 0.f;
#pragma unroll
    for (int c = 0; c < CMAX; c++)
      if (c < d.C) {
        acc[c] = mul4(kid_S(g, k0, c0, c, l0[c]), kid_S(g, k1, c1, c, l1[c]));
        m = fmaxf(m, fmaxf(fmaxf(acc[c].x, acc[c].y), fmaxf(acc[c].z, acc[c].w)));
      }
    int e = 0;
    if (!isfinite(m)) {
      atomicOr(g.status, ST_NONFINITE);
    } else if (m > 0.f) {
      frexpf(m, &e);
    }
    double site = 0.0;
#pragma unroll
    for (int c = 0; c < CMAX; c++)
      if (c < d.C) {
        const float4 v = ldexp4(acc[c], e);
        g.part[((size_t)slot * d.C + c) * d.P + p] = v;
        if (u == g.root)
          site += g.catw[c] * ((double)v.x * g.pi[0] + (double)v.y * g.pi[1] +
                               (double)v.z * g.pi[2] + (double)v.w * g.pi[3]);
      }
    g.scale[(size_t)slot * d.P + p] = (int16_t)e;
    if (u == g.root) {
      g.site_log[p] = log(site);
      g.site_inv[p] = site > 0.0 ? 1.0 / site : 0.0;
    }
  }
}

// ---- pre-order -------------------------------------------------------------
// Node u of the level: for its kPP patterns and each category, X for both
// children, U stored for internal children, and G accumulated in registers;
// then per category the CTA sums the 32 accumulators through shared memory.
template <int CMAX>
__global__ void __launch_bounds__(kThr, 2) k4_pre(K4Args g, int off) {
  __shared__ float ws[kThr / 32][32][33];  // [warp][value][lane], rows padded
  __shared__ float wsum[kThr / 32][32];
  const Dims &d = g.d;
  const int u = g.nodes[off + blockIdx.y];
  const int slot = u - d.N;
  const bool is_root = (u == g.root);
  // cherries are stored in this pass (their children are tips)
  const int x0 = g.child[2 * slot], x1 = g.child[2 * slot + 1];
  Kid k0 = classify(g, x0), k1 = classify(g, x1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int pj[kPP], e[kPP];
  float n[kPP], sinv[kPP];
  KidCodes cc0[kPP], cc1[kPP];
#pragma unroll
  for (int j = 0; j < kPP; j++) {
    const int p = blockIdx.x * kK4Tile + j * kThr + threadIdx.x;
    const bool act = p < d.P;
    pj[j] = act ? p : 0;
    e[j] = g.scale[(size_t)slot * d.P + pj[j]];
    n[j] = act ? (float)g.pw[pj[j]] : 0.f;
    sinv[j] = is_root ? (float)g.site_inv[pj[j]] : 0.f;
    cc0[j] = kid_codes(g, k0, pj[j]);
    cc1[j] = kid_codes(g, k1, pj[j]);
  }
  for (int c = 0; c < d.C; c++) {
    float4 uu[kPP], L0[kPP], L1[kPP];
#pragma unroll
    for (int j = 0; j < kPP; j++) {
      if (is_root) {
        const float wc = (float)g.catw[c] * sinv[j];
        uu[j] = make_float4(wc * (float)g.pi[0], wc * (float)g.pi[1], wc * (float)g.pi[2],
                            wc * (float)g.pi[3]);
      } else {
        uu[j] = __ldg(g.pre + ((size_t)slot * d.C + c) * d.P + pj[j]);
      }
      L0[j] = kid_L(g, k0, cc0[j], c, pj[j]);
      L1[j] = kid_L(g, k1, cc1[j], c, pj[j]);
    }
    float acc[32];
#pragma unroll
    for (int q = 0; q < 32; q++) acc[q] = 0.f;
#pragma unroll
    for (int j = 0; j < kPP; j++) {
      const float4 S0 = kid_S(g, k0, cc0[j], c, L0[j]);
      const float4 S1 = kid_S(g, k1, cc1[j], c, L1[j]);
      const float4 X0 = ldexp4(mul4(uu[j], S1), e[j]);
      const float4 X1 = ldexp4(mul4(uu[j], S0), e[j]);
      const bool act = blockIdx.x * kK4Tile + j * kThr + threadIdx.x < d.P;
      if (act && k0.kind != 0)
        g.pre[((size_t)(x0 - d.N) * d.C + c) * d.P + pj[j]] = matvec(tab(g, x0, c), X0);
      if (act && k1.kind != 0)
        g.pre[((size_t)(x1 - d.N) * d.C + c) * d.P + pj[j]] = matvec(tab(g, x1, c), X1);
      const float xa[4] = {X0.x * n[j], X0.y * n[j], X0.z * n[j], X0.w * n[j]};
      const float xb[4] = {X1.x * n[j], X1.y * n[j], X1.z * n[j], X1.w * n[j]};
      const float la[4] = {L0[j].x, L0[j].y, L0[j].z, L0[j].w};
      const float lb[4] = {L1[j].x, L1[j].y, L1[j].z, L1[j].w};
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int jj = 0; jj < 4; jj++) {
          acc[i * 4 + jj] += xa[i] * la[jj];
          acc[16 + i * 4 + jj] += xb[i] * lb[jj];
        }
    }
    // warp transpose: lane l sums value l over the warp's lanes
#pragma unroll
    for (int q = 0; q < 32; q++) ws[warp][q][lane] = acc[q];
    __syncwarp();
    float t = 0.f;
#pragma unroll
    for (int l = 0; l < 32; l++) t += ws[warp][lane][l];
    wsum[warp][lane] = t;
    __syncthreads();
    if (warp == 0) {
      float s = 0.f;
      for (int w = 0; w < kThr / 32; w++) s += wsum[w][lane];
      const int br = (lane < 16) ? x0 : x1;
      g.Gpart[(((size_t)br * g.ntile + blockIdx.x) * d.C + c) * 16 + (lane & 15)] = s;
    }
    __syncthreads();
  }
}

// Cherries in the pre-order pass: U of the cherry is stored by its parent;
// here X for its two tips and their G (tips: indicator vectors).
template <int CMAX>
__global__ void __launch_bounds__(kThr, 2) k4_pre_cherry(K4Args g, int off) {
  __shared__ float ws[kThr / 32][32][33];
  __shared__ float wsum[kThr / 32][32];
  const Dims &d = g.d;
  const int u = g.nodes[off + blockIdx.y];
  const int slot = u - d.N;
  const int a = g.child[2 * slot], b = g.child[2 * slot + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int pj[kPP], ca[kPP], cb[kPP];
  float n[kPP];
#pragma unroll
  for (int j = 0; j < kPP; j++) {
    const int p = blockIdx.x * kK4Tile + j * kThr + threadIdx.x;
    const bool act = p < d.P;
    pj[j] = act ? p : 0;
    n[j] = act ? (float)g.pw[pj[j]] : 0.f;
    ca[j] = g.tips[(size_t)a * d.P + pj[j]];
    cb[j] = g.tips[(size_t)b * d.P + pj[j]];
  }
  for (int c = 0; c < d.C; c++) {
    float4 uu[kPP];
#pragma unroll
    for (int j = 0; j < kPP; j++) uu[j] = __ldg(g.pre + ((size_t)slot * d.C + c) * d.P + pj[j]);
    float acc[32];
#pragma unroll
    for (int q = 0; q < 32; q++) acc[q] = 0.f;
#pragma unroll
    for (int j = 0; j < kPP; j++) {
      const float4 Sa = __ldg(tab(g, a, c) + ca[j]), Sb = __ldg(tab(g, b, c) + cb[j]);
      const float4 Xa = mul4(uu[j], Sb), Xb = mul4(uu[j], Sa);  // exponent 0
      const float4 oa = onehot(ca[j], g.masks), ob = onehot(cb[j], g.masks);
      const float xa[4] = {Xa.x * n[j], Xa.y * n[j], Xa.z * n[j], Xa.w * n[j]};
      const float xb[4] = {Xb.x * n[j], Xb.y * n[j], Xb.z * n[j], Xb.w * n[j]};
      const float la[4] = {oa.x, oa.y, oa.z, oa.w};
      const float lb[4] = {ob.x, ob.y, ob.z, ob.w};
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int jj = 0; jj < 4; jj++) {
          acc[i * 4 + jj] += xa[i] * la[jj];
          acc[16 + i * 4 + jj] += xb[i] * lb[jj];
        }
    }
#pragma unroll
    for (int q = 0; q < 32; q++) ws[warp][q][lane] = acc[q];
    __syncwarp();
    float t = 0.f;
#pragma unroll
    for (int l = 0; l < 32; l++) t += ws[warp][lane][l];
    wsum[warp][lane] = t;
    __syncthreads();
    if (warp == 0) {
      float s = 0.f;
      for (int w = 0; w < kThr / 32; w++) s += wsum[w][lane];
      const int br = (lane < 16) ? a : b;
      g.Gpart[(((size_t)br * g.ntile + blockIdx.x) * d.C + c) * 16 + (lane & 15)] = s;
    }
    __syncthreads();
  }
}

// G[v][c][ij] = sum over tiles of branch v's tile sums, FP64, fixed order.
// One warp per (v, c): lanes split the tiles, then a shuffle tree.
__global__ void k4_G_reduce(Dims d, int ntile, const int *__restrict__ parent,
                            const float *__restrict__ Gpart, double *__restrict__ G) {
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (wid >= d.nn * d.C) return;
  const int v = wid / d.C, c = wid % d.C;
  const int ij = lane & 15, half = lane >> 4;
  double acc = 0.0;
  if (parent[v] >= 0)
    for (int t = half; t < ntile; t += 2)
      acc += (double)Gpart[(((size_t)v * ntile + t) * d.C + c) * 16 + ij];
  acc += __shfl_xor_sync(0xffffffffu, acc, 16);
  if (half == 0) G[((size_t)v * d.C + c) * 16 + ij] = acc;
}

// lnL_p = log(scaled root sum) + ln2 * sum_u e_u(p); block sums of n_p lnL_p
// reduced in a fixed order by the last block to finish.
__global__ void __launch_bounds__(256) k4_site_lnl(Dims d, const int16_t *__restrict__ scale,
                                                   const double *__restrict__ site_log,
                                                   const double *__restrict__ pw,
                                                   double *__restrict__ site_lnl,
                                                   double *__restrict__ part, int *ctl,
                                                   double *__restrict__ lnl) {
  __shared__ int es[8][32];
  __shared__ double red[8];
  __shared__ int s_last;
  const int pl = threadIdx.x & 31, gi = threadIdx.x >> 5;
  const int p = blockIdx.x * 32 + pl;
  int acc = 0;
  if (p < d.P)
    for (int s = gi; s < d.N - 1; s += 8) acc += scale[(size_t)s * d.P + p];
  es[gi][pl] = acc;
  __syncthreads();
  double contrib = 0.0;
  if (gi == 0 && p < d.P) {
    int tot = 0;
    for (int k = 0; k < 8; k++) tot += es[k][pl];
    const double lp = site_log[p] + 0.69314718055994530942 * (double)tot;
    site_lnl[p] = lp;
    const double nw = pw[p];
    contrib = (nw != 0.0) ? nw * lp : 0.0;
  }
  if (gi == 0) {
    for (int o = 16; o > 0; o >>= 1) contrib += __shfl_xor_sync(0xffffffffu, contrib, o);
    if (pl == 0) {
      part[blockIdx.x] = contrib;
      __threadfence();
      s_last = (atomicAdd(ctl, 1) == (int)gridDim.x - 1);
    }
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double t = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += __ldcg(part + i);
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (pl == 0) red[gi] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < 8; k++) s += red[k];
    lnl[0] = s;
  }
}

K4Args make_args(epoch_ctx *c) {
  K4Args a;
  a.d = c->d;
  a.PT = reinterpret_cast<const float4 *>(c->d_PT32);
  a.nodes = c->d_level_nodes;
  a.child = c->d_child;
  a.part = reinterpret_cast<float4 *>(c->d_part);
  a.pre = reinterpret_cast<float4 *>(c->d_pre);
  a.scale = c->d_scale;
  a.tips = c->d_tips;
  a.masks = c->d_masks;
  a.pi = c->d_pi;
  a.catw = c->d_catw;
  a.pw = c->d_pw;
  a.root = c->root;
  a.site_log = c->d_site_log;
  a.site_inv = c->d_site_inv;
  a.Gpart = (float *)c->d_Gpart;
  a.ntile = ceil_div(c->d.P, kK4Tile);
  a.status = c->d_status;
  return a;
}

template <int CMAX>
cudaError_t post(epoch_ctx *c) {
  K4Args a = make_args(c);
  const int L = (int)c->h_level_off.size() - 1;
  for (int l = c->k4_first_level; l < L; l++) {
    const int w = c->h_level_off[l + 1] - c->h_level_off[l];
    k4_post<CMAX><<<dim3(ceil_div(c->d.P, kThr), w), kThr, 0, c->stream>>>(a, c->h_level_off[l]);
    c->launches++;
  }
  cudaMemsetAsync(c->d_ctl, 0, sizeof(int), c->stream);
  k4_site_lnl<<<ceil_div(c->d.P, 32), 256, 0, c->stream>>>(c->d, c->d_scale, c->d_site_log,
                                                           c->d_pw, c->d_site_lnl,
                                                           c->d_lnl_part, c->d_ctl, c->d_lnl);
  c->launches++;
  return cudaGetLastError();
}

template <int CMAX>
cudaError_t pre(epoch_ctx *c) {
  K4Args a = make_args(c);
  const int L = (int)c->h_level_off.size() - 1;
  for (int l = L - 1; l >= c->k4_first_level; l--) {
    const int w = c->h_level_off[l + 1] - c->h_level_off[l];
    k4_pre<CMAX><<<dim3(a.ntile, w), kThr, 0, c->stream>>>(a, c->h_level_off[l]);
    c->launches++;
  }
  if (c->k4_first_level == 1) {  // the cherries
    const int w = c->h_level_off[1] - c->h_level_off[0];
    k4_pre_cherry<CMAX><<<dim3(a.ntile, w), kThr, 0, c->stream>>>(a, c->h_level_off[0]);
    c->launches++;
  }
  const int warps = c->d.nn * c->d.C;
  k4_G_reduce<<<ceil_div(warps * 32, 256), 256, 0, c->stream>>>(c->d, a.ntile, c->d_parent,
                                                                (const float *)c->d_Gpart, c->d_G);
  c->launches++;
  return cudaGetLastError();
}

}  // namespace

int k4_tile() { return kK4Tile; }

cudaError_t launch_partials_k4(epoch_ctx *c) {
  if (c->d.C <= 4) return post<4>(c);
  if (c->d.C <= 8) return post<8>(c);
  return post<16>(c);
}

cudaError_t launch_preorder_k4(epoch_ctx *c) {
  if (c->d.C <= 4) return pre<4>(c);
  if (c->d.C <= 8) return pre<8>(c);
  return pre<16>(c);
}

}  // namespace epoch
