// k_k4.cu -- the FP32 path for K = 4 (nucleotides): post-order pruning with
// rescaling, and the pre-order adjoint pass with the per-branch adjoint G.
//
//  * One launch per post-order level; grid = (tiles of 256 patterns, nodes
//    of the level).  The 16-byte state vector of a (category, pattern) is one
//    load; every branch table a CTA needs sits in shared memory.
//  * Cherries (internal nodes whose two children are tips) are not stored by
//    the post-order pass.  Their partial L = T_a[code_a] o T_b[code_b] and
//    S = P L depend only on the pair of one-byte tip codes, so k4_pair_tables
//    tabulates both for every code pair (NR^2 entries per category, NR = K +
//    1 + masks) right after the branch matrices; a parent then reads a
//    cherry child's S (and, in the adjoint, its L) with one lookup.  A
//    cherry's values are products of probabilities: no rescaling (e = 0).
//    The pre-order pass stores every internal node's outside partial U,
//    cherries included, and visits the cherries' level too, so each node's
//    step touches exactly its two child branches.
//  * Power-of-two rescaling by exponent arithmetic (exact).
//  * Adjoint threads are laid out as (category, pattern lane); a thread owns
//    kPPT patterns of one category, keeps the 32 G accumulators of its two
//    branches in registers, and the CTA reduces them once, through shared
//    memory in a fixed order (deterministic), into a per-(branch, tile)
//    sum; k4_G_reduce adds the tiles in FP64.
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "epoch_internal.cuh"

namespace epoch {
namespace {

constexpr int kThr = 256;  // threads per CTA
constexpr int kTP = 256;   // patterns per CTA tile
constexpr int kBatch = 2;  // adjoint patterns whose loads are issued together

__device__ __forceinline__ float4 mul4(float4 a, float4 b) {
  return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w);
}
__device__ __forceinline__ float4 scl4(float4 a, float s) {
  return make_float4(a.x * s, a.y * s, a.z * s, a.w * s);
}
__device__ __forceinline__ float dot4(float4 a, float4 b) {
  return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
}
// a * 2^-e, exact; e is the binary exponent of a value in (0, 2] so -e is in
// [-1, 149]: one multiply by 2^-e when -e <= 126, else by 2^126 then 2^(-e-126).
__device__ __forceinline__ float4 pow2_scale(float4 a, int e) {
  if (e >= -126) return scl4(a, __int_as_float((127 - e) << 23));
  return scl4(scl4(a, __int_as_float(253 << 23)), __int_as_float((1 - e) << 23));
}
// S = P L with rows t[j] = column j of P: S = sum_j L_j t[j]
__device__ __forceinline__ float4 matvec_t(const float4 *t, float4 l) {
  const float4 r0 = t[0], r1 = t[1], r2 = t[2], r3 = t[3];
  float4 s;
  s.x = l.x * r0.x + l.y * r1.x + l.z * r2.x + l.w * r3.x;
  s.y = l.x * r0.y + l.y * r1.y + l.z * r2.y + l.w * r3.y;
  s.z = l.x * r0.z + l.y * r1.z + l.z * r2.z + l.w * r3.z;
  s.w = l.x * r0.w + l.y * r1.w + l.z * r2.w + l.w * r3.w;
  return s;
}
// U = P^T X: U_j = <t[j], X>
__device__ __forceinline__ float4 matvec(const float4 *t, float4 x) {
  return make_float4(dot4(t[0], x), dot4(t[1], x), dot4(t[2], x), dot4(t[3], x));
}
__device__ __forceinline__ float4 onehot(int code, const unsigned long long *masks) {
  const unsigned long long mk = code < 4 ? (1ull << code) : (code == 4 ? ~0ull : masks[code - 5]);
  return make_float4((mk & 1ull) ? 1.f : 0.f, (mk & 2ull) ? 1.f : 0.f, (mk & 4ull) ? 1.f : 0.f,
                     (mk & 8ull) ? 1.f : 0.f);
}

struct K4Args {
  Dims d;
  const float4 *PT;        // [nn][C][NR] rows of Kp = 4 floats
  const float4 *pairS;     // [nn][C][NR*NR] S of a cherry for each code pair
  const float4 *pairL;     // [nn][C][NR*NR] L of a cherry for each code pair
  const int *nodes;        // internal nodes, level-ascending
  const int *child;        // [N-1][2]
  float4 *part;            // [N-1][C][P]
  float4 *pre;             // [N-1][C][P]
  int16_t *scale;          // [N-1][Pp]
  const uint8_t *tips;     // [N][Pp]
  const unsigned long long *masks;
  const double *pi, *catw;
  const float *pwf;        // [Pp]
  int root;
  double *site_log, *site_inv;
  float *Gpart;            // [nn][tiles][C][16]
  int ntile;
  int *status;
};

// A child: kind 0 tip, 1 cherry (tips a, b), 2 stored.
struct Kid {
  int node, kind, a, b;
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

// ---- pair tables of the cherries --------------------------------------------
// One CTA per internal node (non-cherries return); threads over (c, pair).
__global__ void k4_pair_tables(Dims d, const float4 *__restrict__ PT, const int *__restrict__ child,
                               int root, float4 *__restrict__ pairS, float4 *__restrict__ pairL) {
  const int u = d.N + blockIdx.x;
  const int a = child[2 * blockIdx.x], b = child[2 * blockIdx.x + 1];
  if (a >= d.N || b >= d.N || u == root) return;
  const int NR = d.NR, NR2 = NR * NR;
  for (int idx = threadIdx.x; idx < d.C * NR2; idx += blockDim.x) {
    const int c = idx / NR2, pr = idx % NR2, ca = pr / NR, cb = pr % NR;
    const float4 L = mul4(PT[((size_t)a * d.C + c) * NR + ca], PT[((size_t)b * d.C + c) * NR + cb]);
    const float4 S = matvec_t(PT + ((size_t)u * d.C + c) * NR, L);
    pairL[((size_t)u * d.C + c) * NR2 + pr] = L;
    pairS[((size_t)u * d.C + c) * NR2 + pr] = S;
  }
}

// Shared-memory tables of one child for all categories.
//   tip:    rows [C][NR]          (S = row[code])
//   cherry: S pairs [C][NR2], then L pairs [C][NR2] (pre-order only), then
//           the first 4 rows [C][4] of its own table (pre-order: U = P^T X)
//   stored: first 4 rows [C][4]
__device__ __forceinline__ int table_size(const K4Args &g, const Kid &k, bool pre) {
  const int C = g.d.C, NR = g.d.NR;
  if (k.kind == 0) return C * NR;
  if (k.kind == 1) return pre ? C * (2 * NR * NR + 4) : C * NR * NR;
  return C * 4;
}
__device__ void load_table(const K4Args &g, const Kid &k, bool pre, float4 *dst) {
  const int C = g.d.C, NR = g.d.NR, NR2 = NR * NR;
  if (k.kind == 0) {
    for (int i = threadIdx.x; i < C * NR; i += blockDim.x) dst[i] = g.PT[(size_t)k.node * C * NR + i];
  } else if (k.kind == 1) {
    for (int i = threadIdx.x; i < C * NR2; i += blockDim.x) dst[i] = g.pairS[(size_t)k.node * C * NR2 + i];
    if (pre) {
      for (int i = threadIdx.x; i < C * NR2; i += blockDim.x)
        dst[C * NR2 + i] = g.pairL[(size_t)k.node * C * NR2 + i];
      for (int i = threadIdx.x; i < C * 4; i += blockDim.x)
        dst[2 * C * NR2 + i] = g.PT[((size_t)k.node * C + i / 4) * NR + (i & 3)];
    }
  } else {
    for (int i = threadIdx.x; i < C * 4; i += blockDim.x)
      dst[i] = g.PT[((size_t)k.node * C + i / 4) * NR + (i & 3)];
  }
}

// ---- post-order ------------------------------------------------------------
template <int CMAX>
__global__ void __launch_bounds__(kThr) k4_post(K4Args g, int off) {
  extern __shared__ float4 tabs[];
  const Dims &d = g.d;
  const int C = d.C, NR = d.NR, NR2 = NR * NR;
  const int u = g.nodes[off + blockIdx.y];
  const int slot = u - d.N;
  const Kid k0 = classify(g, g.child[2 * slot]), k1 = classify(g, g.child[2 * slot + 1]);
  float4 *t0 = tabs, *t1 = tabs + table_size(g, k0, false);
  load_table(g, k0, false, t0);
  load_table(g, k1, false, t1);
  const int p = blockIdx.x * kTP + threadIdx.x;
  // loads first (stored children's vectors, codes), then the tables barrier
  float4 l0[CMAX], l1[CMAX];
  int i0 = 0, i1 = 0;
  if (p < d.P) {
    if (k0.kind == 2) {
#pragma unroll
      for (int c = 0; c < CMAX; c++)
        if (c < C) l0[c] = __ldcs(g.part + ((size_t)(k0.node - d.N) * C + c) * d.P + p);
    } else if (k0.kind == 1) {
      i0 = g.tips[(size_t)k0.a * d.Pp + p] * NR + g.tips[(size_t)k0.b * d.Pp + p];
    } else {
      i0 = g.tips[(size_t)k0.node * d.Pp + p];
    }
    if (k1.kind == 2) {
#pragma unroll
      for (int c = 0; c < CMAX; c++)
        if (c < C) l1[c] = __ldcs(g.part + ((size_t)(k1.node - d.N) * C + c) * d.P + p);
    } else if (k1.kind == 1) {
      i1 = g.tips[(size_t)k1.a * d.Pp + p] * NR + g.tips[(size_t)k1.b * d.Pp + p];
    } else {
      i1 = g.tips[(size_t)k1.node * d.Pp + p];
    }
  }
  __syncthreads();
  if (p >= d.P) return;
  float4 acc[CMAX];
  float m = 0.f;
#pragma unroll
  for (int c = 0; c < CMAX; c++)
    if (c < C) {
      const float4 s0 = k0.kind == 2 ? matvec_t(t0 + 4 * c, l0[c])
                                     : t0[k0.kind == 1 ? c * NR2 + i0 : c * NR + i0];
      const float4 s1 = k1.kind == 2 ? matvec_t(t1 + 4 * c, l1[c])
                                     : t1[k1.kind == 1 ? c * NR2 + i1 : c * NR + i1];
      acc[c] = mul4(s0, s1);
      m = fmaxf(m, fmaxf(fmaxf(acc[c].x, acc[c].y), fmaxf(acc[c].z, acc[c].w)));
    }
  int e = 0;
  if (!(m <= 3.0e38f)) {  // NaN or Inf
    atomicOr(g.status, ST_NONFINITE);
  } else if (m > 0.f) {
    e = ((__float_as_int(m) >> 23) & 255) - 126;  // m = f 2^e, f in [0.5, 1)
    if (e == -126) frexpf(m, &e);                 // denormal maximum
  }
  double site = 0.0;
#pragma unroll
  for (int c = 0; c < CMAX; c++)
    if (c < C) {
      const float4 v = pow2_scale(acc[c], e);
      g.part[((size_t)slot * C + c) * d.P + p] = v;
      if (u == g.root)
        site += g.catw[c] * ((double)v.x * g.pi[0] + (double)v.y * g.pi[1] +
                             (double)v.z * g.pi[2] + (double)v.w * g.pi[3]);
    }
  g.scale[(size_t)slot * d.Pp + p] = (int16_t)e;
  if (u == g.root) {
    g.site_log[p] = log(site);
    g.site_inv[p] = site > 0.0 ? 1.0 / site : 0.0;
  }
}

// ---- pre-order -------------------------------------------------------------
// Thread = (category c, lane): c = tid / GS, GS = kThr / Cp; the thread owns
// patterns lane + GS k of the tile (Cp of them), processed kBatch at a
// time with their loads issued together.
template <int CMAX>
__global__ void __launch_bounds__(kThr, 2) k4_pre(K4Args g, int off, int Cp) {
  extern __shared__ float4 tabs[];
  __shared__ float red[kThr / 32][32][33];
  __shared__ float wsum[kThr / 32][32];
  const Dims &d = g.d;
  const int C = d.C, NR = d.NR, NR2 = NR * NR;
  const int u = g.nodes[off + blockIdx.y];
  const int slot = u - d.N;
  const bool is_root = (u == g.root);
  const int x0 = g.child[2 * slot], x1 = g.child[2 * slot + 1];
  const Kid k0 = classify(g, x0), k1 = classify(g, x1);
  float4 *t0 = tabs, *t1 = tabs + table_size(g, k0, true);
  load_table(g, k0, true, t0);
  load_table(g, k1, true, t1);
  const int GS = kThr / Cp;
  const int c = threadIdx.x / GS, lp = threadIdx.x % GS;
  const bool cact = c < C;
  const int cc = cact ? c : 0;
  const float wc = (float)g.catw[cc];
  const float4 pi4 = make_float4((float)g.pi[0], (float)g.pi[1], (float)g.pi[2], (float)g.pi[3]);
  __syncthreads();
  // this category's table views
  const float4 *S0t = k0.kind == 0 ? t0 + cc * NR : (k0.kind == 1 ? t0 + cc * NR2 : nullptr);
  const float4 *S1t = k1.kind == 0 ? t1 + cc * NR : (k1.kind == 1 ? t1 + cc * NR2 : nullptr);
  const float4 *L0t = k0.kind == 1 ? t0 + C * NR2 + cc * NR2 : nullptr;
  const float4 *L1t = k1.kind == 1 ? t1 + C * NR2 + cc * NR2 : nullptr;
  const float4 *P0 = k0.kind == 0 ? t0 + cc * NR : (k0.kind == 1 ? t0 + 2 * C * NR2 + 4 * cc : t0 + 4 * cc);
  const float4 *P1 = k1.kind == 0 ? t1 + cc * NR : (k1.kind == 1 ? t1 + 2 * C * NR2 + 4 * cc : t1 + 4 * cc);
  float acc[32];
#pragma unroll
  for (int q = 0; q < 32; q++) acc[q] = 0.f;
  const int p0 = blockIdx.x * kTP;
  if (cact) {
    for (int kb = 0; kb < Cp; kb += kBatch) {
      float4 uu[kBatch], L0[kBatch], L1[kBatch];
      int e[kBatch], i0[kBatch], i1[kBatch];
      float n[kBatch];
      bool act[kBatch];
#pragma unroll
      for (int k = 0; k < kBatch; k++) {
        const int p = p0 + lp + GS * (kb + k);
        act[k] = (kb + k < Cp) && p < d.P;
        const int pc = act[k] ? p : 0;
        e[k] = g.scale[(size_t)slot * d.Pp + pc];
        n[k] = act[k] ? g.pwf[pc] : 0.f;
        if (is_root) {
          const float w = wc * (float)g.site_inv[pc];
          uu[k] = make_float4(w * pi4.x, w * pi4.y, w * pi4.z, w * pi4.w);
        } else {
          uu[k] = __ldg(g.pre + ((size_t)slot * C + cc) * d.P + pc);
        }
        if (k0.kind == 2) L0[k] = __ldg(g.part + ((size_t)(x0 - d.N) * C + cc) * d.P + pc);
        else if (k0.kind == 1) i0[k] = g.tips[(size_t)k0.a * d.Pp + pc] * NR + g.tips[(size_t)k0.b * d.Pp + pc];
        else i0[k] = g.tips[(size_t)x0 * d.Pp + pc];
        if (k1.kind == 2) L1[k] = __ldg(g.part + ((size_t)(x1 - d.N) * C + cc) * d.P + pc);
        else if (k1.kind == 1) i1[k] = g.tips[(size_t)k1.a * d.Pp + pc] * NR + g.tips[(size_t)k1.b * d.Pp + pc];
        else i1[k] = g.tips[(size_t)x1 * d.Pp + pc];
      }
#pragma unroll
      for (int k = 0; k < kBatch; k++) {
        if (k0.kind == 1) L0[k] = L0t[i0[k]];
        else if (k0.kind == 0) L0[k] = onehot(i0[k], g.masks);
        if (k1.kind == 1) L1[k] = L1t[i1[k]];
        else if (k1.kind == 0) L1[k] = onehot(i1[k], g.masks);
        const float4 S0 = k0.kind == 2 ? matvec_t(P0, L0[k]) : S0t[i0[k]];
        const float4 S1 = k1.kind == 2 ? matvec_t(P1, L1[k]) : S1t[i1[k]];
        const float4 X0 = pow2_scale(mul4(uu[k], S1), e[k]);
        const float4 X1 = pow2_scale(mul4(uu[k], S0), e[k]);
        const int p = p0 + lp + GS * (kb + k);
        if (act[k] && k0.kind != 0) g.pre[((size_t)(x0 - d.N) * C + cc) * d.P + p] = matvec(P0, X0);
        if (act[k] && k1.kind != 0) g.pre[((size_t)(x1 - d.N) * C + cc) * d.P + p] = matvec(P1, X1);
        const float xa[4] = {X0.x * n[k], X0.y * n[k], X0.z * n[k], X0.w * n[k]};
        const float xb[4] = {X1.x * n[k], X1.y * n[k], X1.z * n[k], X1.w * n[k]};
        const float la[4] = {L0[k].x, L0[k].y, L0[k].z, L0[k].w};
        const float lb[4] = {L1[k].x, L1[k].y, L1[k].z, L1[k].w};
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
          for (int j = 0; j < 4; j++) {
            acc[i * 4 + j] += xa[i] * la[j];
            acc[16 + i * 4 + j] += xb[i] * lb[j];
          }
      }
    }
  }
  // per-warp transpose: lane l sums value l; then the warps of a category
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 32; q++) red[warp][q][lane] = acc[q];
  __syncwarp();
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 32; k++) s += red[warp][lane][k];
  wsum[warp][lane] = s;
  __syncthreads();
  const int wpc = (GS + 31) / 32;
  for (int idx = threadIdx.x; idx < C * 32; idx += blockDim.x) {
    const int cq = idx >> 5, l = idx & 31;
    float tot = 0.f;
    for (int k = 0; k < wpc; k++) tot += wsum[cq * wpc + k][l];
    const int br = (l < 16) ? x0 : x1;
    g.Gpart[(((size_t)br * g.ntile + blockIdx.x) * C + cq) * 16 + (l & 15)] = tot;
  }
}

// G[v][c][ij] = sum over the tiles of branch v, FP64, fixed order.
__global__ void k4_G_reduce(Dims d, int ntile, const int *__restrict__ parent,
                            const float *__restrict__ Gpart, double *__restrict__ G) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)d.nn * d.C * 16) return;
  const int ij = (int)(idx & 15);
  const int c = (int)((idx >> 4) % d.C);
  const int v = (int)(idx / (16LL * d.C));
  double acc = 0.0;
  if (parent[v] >= 0)
#pragma unroll 8
    for (int t = 0; t < ntile; t++)
      acc += (double)Gpart[(((size_t)v * ntile + t) * d.C + c) * 16 + ij];
  G[idx] = acc;
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
  __shared__ double redd[8];
  __shared__ int s_last;
  const int pl = threadIdx.x & 31, gi = threadIdx.x >> 5;
  const int p = blockIdx.x * 32 + pl;
  int acc = 0;
  if (p < d.P)
#pragma unroll 8
    for (int s = gi; s < d.N - 1; s += 8) acc += scale[(size_t)s * d.Pp + p];
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
  if (pl == 0) redd[gi] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < 8; k++) s += redd[k];
    lnl[0] = s;
  }
}

K4Args make_args(epoch_ctx *c) {
  K4Args a{};
  a.d = c->d;
  a.PT = reinterpret_cast<const float4 *>(c->d_PT32);
  a.pairS = reinterpret_cast<const float4 *>(c->d_pairS);
  a.pairL = reinterpret_cast<const float4 *>(c->d_pairL);
  a.nodes = c->d_level_nodes;
  a.child = c->d_child;
  a.part = reinterpret_cast<float4 *>(c->d_part);
  a.pre = reinterpret_cast<float4 *>(c->d_pre);
  a.scale = c->d_scale;
  a.tips = c->d_tips;
  a.masks = c->d_masks;
  a.pi = c->d_pi;
  a.catw = c->d_catw;
  a.pwf = c->d_pwf;
  a.root = c->root;
  a.site_log = c->d_site_log;
  a.site_inv = c->d_site_inv;
  a.Gpart = (float *)c->d_Gpart;
  a.ntile = ceil_div(c->d.P, kTP);
  a.status = c->d_status;
  return a;
}

// largest table set of a node: two cherry children in the pre-order pass
size_t table_smem(const Dims &d) {
  return sizeof(float4) * 2 * d.C * (2 * d.NR * d.NR + 4);
}

int pow2_at_least(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

template <int CMAX>
cudaError_t post(epoch_ctx *c) {
  K4Args a = make_args(c);
  const int L = (int)c->h_level_off.size() - 1;
  const size_t smem = table_smem(c->d);
  cudaFuncSetAttribute(k4_post<CMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  for (int l = c->k4_first_level; l < L; l++) {
    const int w = c->h_level_off[l + 1] - c->h_level_off[l];
    k4_post<CMAX><<<dim3(a.ntile, w), kThr, smem, c->stream>>>(a, c->h_level_off[l]);
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
  const size_t smem = table_smem(c->d);
  cudaFuncSetAttribute(k4_pre<CMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int Cp = pow2_at_least(c->d.C);
  for (int l = L - 1; l >= 0; l--) {
    const int w = c->h_level_off[l + 1] - c->h_level_off[l];
    k4_pre<CMAX><<<dim3(a.ntile, w), kThr, smem, c->stream>>>(a, c->h_level_off[l], Cp);
    c->launches++;
  }
  const long long nG = (long long)c->d.nn * c->d.C * 16;
  k4_G_reduce<<<ceil_div(nG, 256), 256, 0, c->stream>>>(c->d, a.ntile, c->d_parent,
                                                        (const float *)c->d_Gpart, c->d_G);
  c->launches++;
  return cudaGetLastError();
}

}  // namespace

int k4_tiles(int P) { return (P + kTP - 1) / kTP; }

cudaError_t launch_pair_tables_k4(epoch_ctx *c) {
  if (c->d.N < 2) return cudaSuccess;
  k4_pair_tables<<<c->d.N - 1, 128, 0, c->stream>>>(c->d, reinterpret_cast<const float4 *>(c->d_PT32),
                                                    c->d_child, c->root,
                                                    reinterpret_cast<float4 *>(c->d_pairS),
                                                    reinterpret_cast<float4 *>(c->d_pairL));
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_partials_k4(epoch_ctx *c) {
  if (c->d.C <= 4) return post<4>(c);
  return post<8>(c);
}

cudaError_t launch_preorder_k4(epoch_ctx *c) {
  if (c->d.C <= 4) return pre<4>(c);
  return pre<8>(c);
}

}  // namespace epoch
