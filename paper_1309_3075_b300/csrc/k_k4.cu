// k_k4.cu -- the FP32 path for K = 4 (nucleotides): post-order pruning with
// rescaling, and the pre-order adjoint pass with the per-branch adjoint G.
//
//  * Wide levels of the tree: one launch per post-order level; grid =
//    (pattern tiles, nodes of the level).  The 16-byte state vector of a
//    (category, pattern) is one load; every branch table a CTA needs sits in
//    shared memory.  A CTA branches once on the kinds of its node's two
//    children (tip, cherry, stored) into code specialised for that pair.
//  * The narrow top of the tree (levels of at most kWalkWidth nodes, up to
//    the root) is done by one "walk" launch per pass: every thread owns one
//    (pattern, category) and steps through the top nodes in order, keeping
//    the values its later steps need in its own shared-memory slots.  No
//    thread reads another's values, so the walk has no barriers; patterns
//    are independent (Eq. partial_likelihood), which is what makes this
//    legal.  The host assigns the slots (k4_schedule).
//  * Cherries (internal nodes whose two children are tips) are not stored by
//    the post-order pass.  Their partial L = T_a[code_a] o T_b[code_b] and
//    S = P L depend only on the pair of one-byte tip codes, so
//    k4_pair_tables tabulates both for every code pair (NR^2 entries per
//    category, NR = K + 1 + masks); a parent reads a cherry child's S (and,
//    in the adjoint, its L) with one lookup.  A cherry's values are products
//    of probabilities: no rescaling (e = 0).
//  * Power-of-two rescaling by exponent arithmetic (exact).
//  * Adjoint threads are laid out as (category, pattern lane); a thread owns
//    Cp * m patterns of one category, keeps the 32 G accumulators of its two
//    branches in registers, and the CTA reduces them once, through shared
//    memory in a fixed order (deterministic), into a per-(branch, tile) sum;
//    k4_G_reduce adds the tiles in FP64.  The G of the walk's branches comes
//    from the same kernel with the U stores switched off.
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "epoch_internal.cuh"

namespace epoch {
namespace {

constexpr int kThr = 256;       // threads per CTA of the level kernels
constexpr int kTP = 256;        // patterns of one fine tile
constexpr int kWalkThr = 128;   // threads per CTA of the walks
// widest level the walks take (lnL + gradient of the 500-taxon GTR workload by
// the widest walked level: 1 node 0.433 ms, 2: 0.432, 3: 0.432, 4: 0.448,
// 8: 0.467, 16: 0.502 -- a level kernel over a few nodes already fills more of
// the GPU than the walk's one thread per (pattern, category))
constexpr int kWalkWidth = 2;
constexpr int kWalkSlots = 32;  // value slots per walk thread (16 B each)
constexpr size_t kWalkSmem = 160 * 1024;  // shared memory of a walk CTA at most
enum : int { kTip = 0, kCherry = 1, kStored = 2 };

__device__ __forceinline__ float4 mul4(float4 a, float4 b) {
  return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w);
}
__device__ __forceinline__ float4 scl4(float4 a, float s) {
  return make_float4(a.x * s, a.y * s, a.z * s, a.w * s);
}
__device__ __forceinline__ float dot4(float4 a, float4 b) {
  return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
}
__device__ __forceinline__ float max4(float4 a) {
  return fmaxf(fmaxf(a.x, a.y), fmaxf(a.z, a.w));
}
// a * 2^-e, exact; e is the binary exponent of a value in (0, 2] so -e is in
// [-1, 149]: one multiply by 2^-e when -e <= 126, else by 2^126 then 2^(-e-126).
__device__ __forceinline__ float4 pow2_scale(float4 a, int e) {
  if (e >= -126) return scl4(a, __int_as_float((127 - e) << 23));
  return scl4(scl4(a, __int_as_float(253 << 23)), __int_as_float((1 - e) << 23));
}
// m = f 2^e with f in [0.5, 1); 0 for m = 0
__device__ __forceinline__ int binary_exponent(float m) {
  int e = 0;
  if (m > 0.f) {
    e = ((__float_as_int(m) >> 23) & 255) - 126;
    if (e == -126) frexpf(m, &e);  // denormal maximum
  }
  return e;
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
  float4 *part;            // [N-1][C][P]
  float4 *pre;             // [N-1][C][P]
  int16_t *scale;          // [N-1][Pp]
  const uint8_t *tips;     // [N][Pp]
  const unsigned long long *masks;
  const double *pi, *catw;
  const float *pwf;        // [Pp]
  int root;
  double *site_log, *site_inv;
  float *Gpart;            // [nn][gstride][C][16]
  int gstride;             // fine tiles of 256 patterns
  int top_begin;           // level-order index from which the adjoint stores no U
  const int4 *desc;        // [N-1][3] per internal node, level order (k4_schedule)
  const double *pw;        // [P] pattern weights
  double *site_lnl;        // [P] per-pattern lnL
  double *lnl_part;        // per walk CTA: its sum of n_p lnL_p
  double *lnl;             // [1]
  int *esum;               // [P] sum of the level kernels' exponents (zero between passes)
  int *ctl;                // walk CTAs finished (zero between passes)
  int *status;
};

// A child: kind tip, cherry (tips a, b) or stored.
struct Kid {
  int node, kind, a, b;
};
// From its descriptor {kind, node, tip a, tip b} (k4_schedule).
__device__ __forceinline__ Kid kid_of(int4 q) { return Kid{q.y, q.x, q.z, q.w}; }

// ---- pair tables of the cherries --------------------------------------------
// One CTA per internal node (non-cherries return); threads over (c, pair).
__global__ void k4_pair_tables(Dims d, const float4 *__restrict__ PT, const int *__restrict__ child,
                               int root, float4 *__restrict__ pairS, float4 *__restrict__ pairL) {
  pdl_wait();  // the branch tables
  pdl_trigger();
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
  if (k.kind == kTip) return C * NR;
  if (k.kind == kCherry) return pre ? C * (2 * NR * NR + 4) : C * NR * NR;
  return C * 4;
}
// float4 of the largest post-order table set (two cherry children), 16-byte
// aligned start of the post-order stage
__host__ __device__ __forceinline__ int post_tables_f4(const Dims &d) { return 2 * d.C * d.NR * d.NR; }
__device__ void load_table(const K4Args &g, const Kid &k, bool pre, float4 *dst) {
  const int C = g.d.C, NR = g.d.NR, NR2 = NR * NR;
  if (k.kind == kTip) {
    for (int i = threadIdx.x; i < C * NR; i += blockDim.x) dst[i] = g.PT[(size_t)k.node * C * NR + i];
  } else if (k.kind == kCherry) {
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

// ---- cp.async into a thread's own shared-memory stage -----------------------------
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool full) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int n = full ? 16 : 0;  // 0: fill the 16 bytes with zeros, read nothing
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_prev() {
  asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}

// ---- post-order level kernel ---------------------------------------------------
// Thread = pattern (all categories).  A CTA covers m fine tiles of one node:
// its tables are staged once, and the stored children's vectors of the next
// tile are copied into the thread's own shared-memory stage by cp.async while
// it computes the current one (double buffer; a thread reads only what it
// copied, so no barrier).  The host picks m per level so that the grid fits
// the resident CTAs in as few rounds as possible.
// Stage: [buffer 2][child 2][CMAX][kThr] float4.
struct PostSmall {
  int i0, i1;
};

template <int CMAX, int K0, int K1>
__device__ __forceinline__ void post_tiles(const K4Args &g, int u, const Kid &k0, const Kid &k1,
                                           const float4 *t0, const float4 *t1, float4 *stage,
                                           int m) {
  const Dims &d = g.d;
  const int C = d.C, NR = d.NR, NR2 = NR * NR;
  const int slot = u - d.N;
  const float4 *l0p = K0 == kStored ? g.part + (size_t)(k0.node - d.N) * C * d.P : nullptr;
  const float4 *l1p = K1 == kStored ? g.part + (size_t)(k1.node - d.N) * C * d.P : nullptr;
  const uint8_t *c0a = g.tips + (size_t)(K0 == kCherry ? k0.a : k0.node) * d.Pp;
  const uint8_t *c0b = g.tips + (size_t)(K0 == kCherry ? k0.b : 0) * d.Pp;
  const uint8_t *c1a = g.tips + (size_t)(K1 == kCherry ? k1.a : k1.node) * d.Pp;
  const uint8_t *c1b = g.tips + (size_t)(K1 == kCherry ? k1.b : 0) * d.Pp;
  auto sp = [&](int buf, int side, int c) {
    return stage + ((buf * 2 + side) * CMAX + c) * kThr + threadIdx.x;
  };
  auto pat = [&](int j) { return (blockIdx.x * m + j) * kTP + (int)threadIdx.x; };
  auto issue = [&](int j, int buf, PostSmall &nx) {
    const int p = pat(j);
    const bool act = j < m && p < d.P;
    const int pc = act ? p : 0;
#pragma unroll
    for (int c = 0; c < CMAX; c++)
      if (c < C) {
        if constexpr (K0 == kStored) cp_async16(sp(buf, 0, c), l0p + (size_t)c * d.P + pc, act);
        if constexpr (K1 == kStored) cp_async16(sp(buf, 1, c), l1p + (size_t)c * d.P + pc, act);
      }
    if constexpr (K0 == kCherry) nx.i0 = act ? c0a[pc] * NR + c0b[pc] : 0;
    else if constexpr (K0 == kTip) nx.i0 = act ? c0a[pc] : 0;
    if constexpr (K1 == kCherry) nx.i1 = act ? c1a[pc] * NR + c1b[pc] : 0;
    else if constexpr (K1 == kTip) nx.i1 = act ? c1a[pc] : 0;
    cp_async_commit();
  };
  auto compute = [&](int j, int buf, const PostSmall &cur) {
    const int p = pat(j);
    if (j >= m || p >= d.P) return;
    float4 acc[CMAX];
    float mx = 0.f;
#pragma unroll
    for (int c = 0; c < CMAX; c++)
      if (c < C) {
        float4 s0, s1;
        if constexpr (K0 == kStored) s0 = matvec_t(t0 + 4 * c, *sp(buf, 0, c));
        else if constexpr (K0 == kCherry) s0 = t0[c * NR2 + cur.i0];
        else s0 = t0[c * NR + cur.i0];
        if constexpr (K1 == kStored) s1 = matvec_t(t1 + 4 * c, *sp(buf, 1, c));
        else if constexpr (K1 == kCherry) s1 = t1[c * NR2 + cur.i1];
        else s1 = t1[c * NR + cur.i1];
        acc[c] = mul4(s0, s1);
        mx = fmaxf(mx, max4(acc[c]));
      }
    int e = 0;
    if (!(mx <= 3.0e38f)) atomicOr(g.status, ST_NONFINITE);  // NaN or Inf
    else e = binary_exponent(mx);
    float4 *dst = g.part + (size_t)slot * C * d.P + p;
#pragma unroll
    for (int c = 0; c < CMAX; c++)
      if (c < C) dst[(size_t)c * d.P] = pow2_scale(acc[c], e);
    g.scale[(size_t)slot * d.Pp + p] = (int16_t)e;
    atomicAdd(g.esum + p, e);  // exact; the walk adds its own nodes' and clears it
  };
  PostSmall sa{0, 0}, sb{0, 0};
  issue(0, 0, sa);  // the first tile's operands need no tables: before the barrier
  __syncthreads();  // the node's tables are staged
  for (int j = 0; j < m; j += 2) {
    if (j + 1 < m) issue(j + 1, 1, sb);
    else cp_async_commit();  // empty group keeps the count
    cp_async_wait_prev();    // buffer 0's copies have landed
    compute(j, 0, sa);
    if (j + 1 >= m) break;
    if (j + 2 < m) issue(j + 2, 0, sa);
    else cp_async_commit();
    cp_async_wait_prev();    // buffer 1's copies have landed
    compute(j + 1, 1, sb);
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// early = 1: the predecessor wrote none of the tables (see pdl_wait).  The
// root is never a level kernel's node: the post-order walk always ends with
// the root's level.
template <int CMAX>
__global__ void __launch_bounds__(kThr) k4_post(K4Args g, int off, int early, int m) {
  extern __shared__ float4 tabs[];
  if (!early) pdl_wait();
  const int4 *D = g.desc + 3 * (off + blockIdx.y);
  const int u = D[0].x;
  const Kid k0 = kid_of(D[1]), k1 = kid_of(D[2]);
  float4 *t0 = tabs, *t1 = tabs + table_size(g, k0, false);
  float4 *stage = tabs + post_tables_f4(g.d);
  load_table(g, k0, false, t0);
  load_table(g, k1, false, t1);
  if (early) pdl_wait();
  pdl_trigger();
  switch (k0.kind * 3 + k1.kind) {  // uniform over the CTA (post_tiles has a barrier)
    case 0: post_tiles<CMAX, kTip, kTip>(g, u, k0, k1, t0, t1, stage, m); break;
    case 1: post_tiles<CMAX, kTip, kCherry>(g, u, k0, k1, t0, t1, stage, m); break;
    case 2: post_tiles<CMAX, kTip, kStored>(g, u, k0, k1, t0, t1, stage, m); break;
    case 4: post_tiles<CMAX, kCherry, kCherry>(g, u, k0, k1, t0, t1, stage, m); break;
    case 5: post_tiles<CMAX, kCherry, kStored>(g, u, k0, k1, t0, t1, stage, m); break;
    default: post_tiles<CMAX, kStored, kStored>(g, u, k0, k1, t0, t1, stage, m); break;
  }
}

// ---- pre-order level kernel ------------------------------------------------------
// Thread = (category c, lane): c = tid / GS, GS = kThr / Cp; the CTA covers m
// fine tiles and the thread owns patterns lane + GS k of them (Cp m in all),
// kPreB at a time.  The float4 operands of the next kPreB patterns (U of the
// node, partials of stored children) are copied into the thread's own
// shared-memory stage with cp.async while it computes the current ones
// (double buffer; a thread reads only what it copied, so no barrier).
constexpr int kPreB = 2;
constexpr int kStageF4 = 2 * kPreB * 3 * kThr;  // float4 of the stage

struct PreSmall {
  int e, i0, i1;
  float n;
};

template <int K0, int K1>
__device__ __forceinline__ void pre_node(const K4Args &g, int slot, bool is_root, bool store,
                                         const Kid &k0, const Kid &k1, const float4 *t0,
                                         const float4 *t1, const float4 *Ltip, float4 *stage,
                                         int Cp, int m, float (&acc)[32]) {
  const Dims &d = g.d;
  const int C = d.C, NR = d.NR, NR2 = NR * NR;
  const int GS = kThr / Cp;
  const int c = threadIdx.x / GS, lp = threadIdx.x % GS;
  if (c >= C) {  // idle lanes when C is not a power of two (they take the barrier below)
    __syncthreads();
    return;
  }
  const double wcd = g.catw[c];
  const float4 pi4 = make_float4((float)g.pi[0], (float)g.pi[1], (float)g.pi[2], (float)g.pi[3]);
  // this category's table views
  const float4 *S0t = K0 == kTip ? t0 + c * NR : t0 + c * NR2;
  const float4 *S1t = K1 == kTip ? t1 + c * NR : t1 + c * NR2;
  const float4 *L0t = t0 + C * NR2 + c * NR2;
  const float4 *L1t = t1 + C * NR2 + c * NR2;
  const float4 *P0 = K0 == kCherry ? t0 + 2 * C * NR2 + 4 * c : t0 + 4 * c;
  const float4 *P1 = K1 == kCherry ? t1 + 2 * C * NR2 + 4 * c : t1 + 4 * c;
  const float4 *up = g.pre + ((size_t)slot * C + c) * d.P;
  const int16_t *ep = g.scale + (size_t)slot * d.Pp;
  const float4 *l0p = K0 == kStored ? g.part + ((size_t)(k0.node - d.N) * C + c) * d.P : nullptr;
  const float4 *l1p = K1 == kStored ? g.part + ((size_t)(k1.node - d.N) * C + c) * d.P : nullptr;
  float4 *w0p = K0 != kTip ? g.pre + ((size_t)(k0.node - d.N) * C + c) * d.P : nullptr;
  float4 *w1p = K1 != kTip ? g.pre + ((size_t)(k1.node - d.N) * C + c) * d.P : nullptr;
  const uint8_t *c0a = g.tips + (size_t)(K0 == kCherry ? k0.a : k0.node) * d.Pp;
  const uint8_t *c0b = g.tips + (size_t)(K0 == kCherry ? k0.b : 0) * d.Pp;
  const uint8_t *c1a = g.tips + (size_t)(K1 == kCherry ? k1.a : k1.node) * d.Pp;
  const uint8_t *c1b = g.tips + (size_t)(K1 == kCherry ? k1.b : 0) * d.Pp;
  const int npat = Cp * m;
  const int pbase = blockIdx.x * kTP * m + lp;
  // stage[buf][k][operand][thread]
  auto sp = [&](int buf, int k, int o) { return stage + ((buf * kPreB + k) * 3 + o) * kThr + threadIdx.x; };
  // two register sets for the small per-pattern values, used in turn so a
  // set's loads have a whole compute phase to land before they are read
  auto issue = [&](int j0, int buf, PreSmall (&nxt)[kPreB]) {
#pragma unroll
    for (int k = 0; k < kPreB; k++) {
      const int p = pbase + GS * (j0 + k);
      const bool act = (j0 + k < npat) && p < d.P;
      const int pc = act ? p : 0;
      if (!is_root) cp_async16(sp(buf, k, 0), up + pc, act);
      if constexpr (K0 == kStored) cp_async16(sp(buf, k, 1), l0p + pc, act);
      if constexpr (K1 == kStored) cp_async16(sp(buf, k, 2), l1p + pc, act);
      nxt[k].e = act ? ep[pc] : 0;
      nxt[k].n = act ? g.pwf[pc] : 0.f;
      if constexpr (K0 == kCherry) nxt[k].i0 = act ? c0a[pc] * NR + c0b[pc] : 0;
      else if constexpr (K0 == kTip) nxt[k].i0 = act ? c0a[pc] : 0;
      if constexpr (K1 == kCherry) nxt[k].i1 = act ? c1a[pc] * NR + c1b[pc] : 0;
      else if constexpr (K1 == kTip) nxt[k].i1 = act ? c1a[pc] : 0;
    }
    cp_async_commit();
  };
  auto compute = [&](int j0, int buf, const PreSmall (&cur)[kPreB]) {
#pragma unroll
    for (int k = 0; k < kPreB; k++) {
      const int p = pbase + GS * (j0 + k);
      const bool act = (j0 + k < npat) && p < d.P;
      // the root's U is the root distribution over the site likelihood
      const float4 uu = is_root ? (act ? scl4(pi4, (float)(wcd * g.site_inv[p])) : pi4)
                                : *sp(buf, k, 0);
      float4 L0, L1, S0, S1;
      if constexpr (K0 == kTip) {
        L0 = Ltip[cur[k].i0];
        S0 = S0t[cur[k].i0];
      } else if constexpr (K0 == kCherry) {
        L0 = L0t[cur[k].i0];
        S0 = S0t[cur[k].i0];
      } else {
        L0 = *sp(buf, k, 1);
        S0 = matvec_t(P0, L0);
      }
      if constexpr (K1 == kTip) {
        L1 = Ltip[cur[k].i1];
        S1 = S1t[cur[k].i1];
      } else if constexpr (K1 == kCherry) {
        L1 = L1t[cur[k].i1];
        S1 = S1t[cur[k].i1];
      } else {
        L1 = *sp(buf, k, 2);
        S1 = matvec_t(P1, L1);
      }
      const float4 X0 = pow2_scale(mul4(uu, S1), cur[k].e);
      const float4 X1 = pow2_scale(mul4(uu, S0), cur[k].e);
      if constexpr (K0 != kTip)
        if (store && act) w0p[p] = matvec(P0, X0);
      if constexpr (K1 != kTip)
        if (store && act) w1p[p] = matvec(P1, X1);
      const float n = cur[k].n;
      const float xa[4] = {X0.x * n, X0.y * n, X0.z * n, X0.w * n};
      const float xb[4] = {X1.x * n, X1.y * n, X1.z * n, X1.w * n};
      const float la[4] = {L0.x, L0.y, L0.z, L0.w};
      const float lb[4] = {L1.x, L1.y, L1.z, L1.w};
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
          acc[i * 4 + j] += xa[i] * la[j];
          acc[16 + i * 4 + j] += xb[i] * lb[j];
        }
    }
  };
  PreSmall sa[kPreB], sb[kPreB];
  issue(0, 0, sa);  // the first operands need no tables: before the barrier
  __syncthreads();  // the node's tables are staged
  for (int j0 = 0; j0 < npat; j0 += 2 * kPreB) {
    if (j0 + kPreB < npat) issue(j0 + kPreB, 1, sb);
    else cp_async_commit();  // empty group keeps the count
    cp_async_wait_prev();    // buffer 0's copies have landed
    compute(j0, 0, sa);
    if (j0 + kPreB >= npat) break;
    if (j0 + 2 * kPreB < npat) issue(j0 + 2 * kPreB, 0, sa);
    else cp_async_commit();
    cp_async_wait_prev();    // buffer 1's copies have landed
    compute(j0 + kPreB, 1, sb);
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

__global__ void __launch_bounds__(kThr, 2) k4_pre(K4Args g, int off, int Cp, int m) {
  extern __shared__ float4 tabs[];
  __shared__ float red[kThr / 32][32][33];
  __shared__ float wsum[kThr / 32][32];
  const Dims &d = g.d;
  const int C = d.C;
  const int idx = off + blockIdx.y;
  const int4 *D = g.desc + 3 * idx;
  const int u = D[0].x;
  const int slot = u - d.N;
  const bool is_root = (u == g.root), store = idx < g.top_begin;
  const Kid k0 = kid_of(D[1]), k1 = kid_of(D[2]);
  float4 *t0 = tabs, *t1 = tabs + table_size(g, k0, true);
  float4 *Ltip = t1 + table_size(g, k1, true);
  float4 *stage = tabs + 2 * C * (2 * d.NR * d.NR + 4) + d.NR;  // after the largest table set
  load_table(g, k0, true, t0);
  load_table(g, k1, true, t1);
  for (int i = threadIdx.x; i < d.NR; i += blockDim.x) Ltip[i] = onehot(i, g.masks);
  pdl_wait();  // the level above (or the walk) has stored this level's U
  pdl_trigger();
  float acc[32];
#pragma unroll
  for (int q = 0; q < 32; q++) acc[q] = 0.f;
  switch (k0.kind * 3 + k1.kind) {  // uniform over the CTA (pre_node has a barrier)
    case 0: pre_node<kTip, kTip>(g, slot, is_root, store, k0, k1, t0, t1, Ltip, stage, Cp, m, acc); break;
    case 1: pre_node<kTip, kCherry>(g, slot, is_root, store, k0, k1, t0, t1, Ltip, stage, Cp, m, acc); break;
    case 2: pre_node<kTip, kStored>(g, slot, is_root, store, k0, k1, t0, t1, Ltip, stage, Cp, m, acc); break;
    case 4: pre_node<kCherry, kCherry>(g, slot, is_root, store, k0, k1, t0, t1, Ltip, stage, Cp, m, acc); break;
    case 5: pre_node<kCherry, kStored>(g, slot, is_root, store, k0, k1, t0, t1, Ltip, stage, Cp, m, acc); break;
    default: pre_node<kStored, kStored>(g, slot, is_root, store, k0, k1, t0, t1, Ltip, stage, Cp, m, acc); break;
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
  const int GS = kThr / Cp;
  const int wpc = (GS + 31) / 32;
  for (int i = threadIdx.x; i < C * 32; i += blockDim.x) {
    const int cq = i >> 5, l = i & 31;
    float tot = 0.f;
    for (int k = 0; k < wpc; k++) tot += wsum[cq * wpc + k][l];
    const int br = (l < 16) ? k0.node : k1.node;
    g.Gpart[(((size_t)br * g.gstride + blockIdx.x) * C + cq) * 16 + (l & 15)] = tot;
  }
}

// ---- walks over the narrow top of the tree ---------------------------------------
// Step descriptor, four int4 (built by k4_schedule):
//   w[0] = {u, value slot (post: out, pre: in; -1 none), u is the root, 0}
//   w[1], w[2] = the children {kind, node, tip a, tip b}
//   w[3] = {child 0 slot, child 1 slot, 0, 0}  (post: where a stored child's
//          value is; pre: where the child's U goes; -1 = not in the walk)
// Shared memory of a walk CTA: the descriptors [steps][4] int4, the first
// four table rows of every non-tip child [steps][2][C][4] float4, the table
// index of every tip or cherry child for the CTA's patterns [steps][2][NPC]
// int (tip: its code; cherry: code_a NR + code_b), then the value slots
// [slots][kWalkThr] float4.  NPC = kWalkThr / CP patterns per CTA.
// Thread = (pattern pl, category c), lane = pl * CP + c.  A thread loads the
// global operands of step i + kWalkDepth while it computes step i (a register
// ring; the step loop is unrolled by kWalkDepth so the ring is indexed
// statically), so the walk waits on memory only at its start.  The operand of
// a tip or cherry child is its S row itself, found through the staged index.
constexpr int kWalkDepth = 8;

struct WalkOp {
  float4 l0, l1;  // stored child: its partial; tip / cherry: table index in .x
  int e;          // pre-order: scale exponent of u
};

__device__ __forceinline__ float4 walk_load(const K4Args &g, int4 k, bool in_slot, int c, int p,
                                            int idx) {
  const Dims &d = g.d;
  if (k.x == kTip) return __ldg(g.PT + ((size_t)k.y * d.C + c) * d.NR + idx);
  if (k.x == kCherry) return __ldg(g.pairS + ((size_t)k.y * d.C + c) * d.NR * d.NR + idx);
  if (in_slot) return make_float4(0.f, 0.f, 0.f, 0.f);
  return g.part[((size_t)(k.y - d.N) * d.C + c) * d.P + p];
}

template <bool POST, int NPC>
__device__ __forceinline__ void walk_fetch(const K4Args &g, const int4 *sd, const int *codes, int s,
                                           int nsteps, int c, int p, int pl, WalkOp &f) {
  if (s >= nsteps) return;
  const int4 h = sd[4 * s], q0 = sd[4 * s + 1], q1 = sd[4 * s + 2], sl = sd[4 * s + 3];
  f.l0 = walk_load(g, q0, POST && sl.x >= 0, c, p, codes[(2 * s) * NPC + pl]);
  f.l1 = walk_load(g, q1, POST && sl.y >= 0, c, p, codes[(2 * s + 1) * NPC + pl]);
  if (!POST) f.e = g.scale[(size_t)(h.x - g.d.N) * g.d.Pp + p];
}

// S = P_x L_x of child q for category c: a tip's or cherry's prefetched row,
// else the product with its staged first four rows
__device__ __forceinline__ float4 walk_S(int4 q, float4 op, const float4 *rows,
                                         const float4 *slotv) {
  if (q.x != kStored) return op;
  return matvec_t(rows, slotv ? *slotv : op);
}

// Stages the descriptors, the table rows and the tip / cherry indices of the
// CTA's patterns (inputs and tables that no kernel of this pass writes: safe
// before pdl_wait); returns the value slots.
template <int NPC>
__device__ float4 *walk_stage(const K4Args &g, const int4 *__restrict__ W, int nsteps, float4 *sm) {
  const Dims &d = g.d;
  const int C = d.C;
  int4 *sd = reinterpret_cast<int4 *>(sm);
  float4 *rows = sm + 4 * nsteps;
  int *codes = reinterpret_cast<int *>(rows + (size_t)nsteps * 8 * C);
  for (int i = threadIdx.x; i < 4 * nsteps; i += blockDim.x) sd[i] = W[i];
  for (int i = threadIdx.x; i < nsteps * 8 * C; i += blockDim.x) {
    const int s = i / (8 * C), r = i % (8 * C), side = r / (4 * C), cr = r % (4 * C);
    const int4 q = W[4 * s + 1 + side];
    if (q.x != kTip) rows[i] = g.PT[((size_t)q.y * C + cr / 4) * d.NR + (cr & 3)];
  }
  for (int i = threadIdx.x; i < nsteps * 2 * NPC; i += blockDim.x) {
    const int sside = i / NPC, pl = i % NPC;
    const int p = blockIdx.x * NPC + pl;
    const int4 q = W[4 * (sside >> 1) + 1 + (sside & 1)];
    int idx = 0;
    if (p < d.P) {
      if (q.x == kTip) idx = g.tips[(size_t)q.y * d.Pp + p];
      else if (q.x == kCherry) idx = g.tips[(size_t)q.z * d.Pp + p] * d.NR + g.tips[(size_t)q.w * d.Pp + p];
    }
    codes[i] = idx;
  }
  __syncthreads();
  return reinterpret_cast<float4 *>(codes + (size_t)nsteps * 2 * NPC);
}

// The root's per-pattern outputs from its scaled partial v (one category per
// lane, CP lanes per pattern): site = sum_c w_c <pi, v_c>, its inverse and
// its log, in FP32 (relative error ~1e-7, far below the FP32 path's bound);
// returns log(site) (every lane).  Out of line: the walk's step loop is
// unrolled, and the root is its last step.
template <int CP>
__device__ __noinline__ float walk_root_site(const K4Args &g, float4 v, bool act, int c, int p) {
  float site = 0.f;
  if (act)
    site = (float)g.catw[c] * (v.x * (float)g.pi[0] + v.y * (float)g.pi[1] +
                               v.z * (float)g.pi[2] + v.w * (float)g.pi[3]);
#pragma unroll
  for (int o = 1; o < CP; o <<= 1) site += __shfl_xor_sync(0xffffffffu, site, o);
  const float ls = logf(site);
  if (c == 0 && p < g.d.P) {
    g.site_log[p] = (double)ls;
    g.site_inv[p] = site > 0.f ? (double)(1.0f / site) : 0.0;
  }
  return ls;
}

// lnL = sum_p n_p lnL_p over the walk's CTAs: each CTA's sum in a fixed
// order into lnl_part, then the last CTA to finish adds those in order and
// zeroes the counter for the next pass.
__device__ void walk_lnl_reduce(const K4Args &g, double contrib) {
  __shared__ double s_red[kWalkThr / 32];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) contrib += __shfl_xor_sync(0xffffffffu, contrib, o);
  if (lane == 0) s_red[warp] = contrib;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kWalkThr / 32; k++) t += s_red[k];
    g.lnl_part[blockIdx.x] = t;
    __threadfence();
    s_last = (atomicAdd(g.ctl, 1) == (int)gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double t = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += __ldcg(g.lnl_part + i);
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  __syncthreads();  // s_red is reused
  if (lane == 0) s_red[warp] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int k = 0; k < kWalkThr / 32; k++) sum += s_red[k];
    g.lnl[0] = sum;
    *g.ctl = 0;
  }
}

template <int CP>
__global__ void __launch_bounds__(kWalkThr) k4_walk_post(K4Args g, const int4 *__restrict__ W,
                                                         int nsteps) {
  extern __shared__ float4 sm[];
  const Dims &d = g.d;
  const int C = d.C;
  constexpr int NPC = kWalkThr / CP;
  float4 *vals = walk_stage<NPC>(g, W, nsteps, sm);
  pdl_wait();
  pdl_trigger();
  const int4 *sd = reinterpret_cast<const int4 *>(sm);
  const float4 *rows = sm + 4 * nsteps;
  const int *codes = reinterpret_cast<const int *>(rows + (size_t)nsteps * 8 * C);
  const int c = threadIdx.x % CP, pl = threadIdx.x / CP;
  const int p = blockIdx.x * NPC + pl;
  const bool act = c < C && p < d.P;
  const int cc = c < C ? c : 0, pc = p < d.P ? p : 0;
  // lnL_p = log(site) + ln2 sum_u e_u(p): lane 0 of a pattern adds the walk's
  // own exponents to the level kernels' sum
  int esum = 0, ebelow = 0;
  double nw = 0.0;
  if (c == 0 && p < d.P) {  // read early: the level kernels have finished
    ebelow = __ldcg(g.esum + p);
    nw = g.pw[p];
  }
  float lsite = 0.f;
  WalkOp ring[kWalkDepth];
#pragma unroll
  for (int k = 0; k < kWalkDepth; k++) walk_fetch<true, NPC>(g, sd, codes, k, nsteps, cc, pc, pl, ring[k]);
  for (int i0 = 0; i0 < nsteps; i0 += kWalkDepth) {
#pragma unroll
    for (int k = 0; k < kWalkDepth; k++) {
      const int i = i0 + k;
      if (i < nsteps) {
        const WalkOp f = ring[k];
        walk_fetch<true, NPC>(g, sd, codes, i + kWalkDepth, nsteps, cc, pc, pl, ring[k]);
        const int4 h = sd[4 * i], q0 = sd[4 * i + 1], q1 = sd[4 * i + 2], sl = sd[4 * i + 3];
        const float4 *r0 = rows + (size_t)i * 8 * C + 4 * cc;
        const float4 *r1 = r0 + 4 * C;
        const float4 s0 = walk_S(q0, f.l0, r0, sl.x >= 0 ? vals + sl.x * kWalkThr + threadIdx.x : nullptr);
        const float4 s1 = walk_S(q1, f.l1, r1, sl.y >= 0 ? vals + sl.y * kWalkThr + threadIdx.x : nullptr);
        const float4 acc = act ? mul4(s0, s1) : make_float4(0.f, 0.f, 0.f, 0.f);
        float mx = max4(acc);
#pragma unroll
        for (int o = 1; o < CP; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        int e = 0;
        if (!(mx <= 3.0e38f)) {
          if (c == 0) atomicOr(g.status, ST_NONFINITE);
        } else {
          e = binary_exponent(mx);
        }
        const float4 v = pow2_scale(acc, e);
        const int slot = h.x - d.N;
        if (act) g.part[((size_t)slot * C + c) * d.P + p] = v;
        if (c == 0 && p < d.P) g.scale[(size_t)slot * d.Pp + p] = (int16_t)e;
        if (c == 0) esum += e;
        if (h.z) {
          lsite = walk_root_site<CP>(g, v, act, c, p);
        } else if (h.y >= 0) {
          vals[h.y * kWalkThr + threadIdx.x] = v;
        }
      }
    }
  }
  double contrib = 0.0;
  if (c == 0 && p < d.P) {
    esum += ebelow;
    g.esum[p] = 0;  // ready for the next pass
    const double lp = (double)lsite + 0.69314718055994530942 * (double)esum;
    g.site_lnl[p] = lp;
    contrib = (nw != 0.0) ? nw * lp : 0.0;
  }
  walk_lnl_reduce(g, contrib);
}

template <int CP>
__global__ void __launch_bounds__(kWalkThr) k4_walk_pre(K4Args g, const int4 *__restrict__ W,
                                                        int nsteps) {
  extern __shared__ float4 sm[];
  const Dims &d = g.d;
  const int C = d.C;
  constexpr int NPC = kWalkThr / CP;
  float4 *vals = walk_stage<NPC>(g, W, nsteps, sm);
  pdl_wait();
  pdl_trigger();
  const int4 *sd = reinterpret_cast<const int4 *>(sm);
  const float4 *rows = sm + 4 * nsteps;
  const int *codes = reinterpret_cast<const int *>(rows + (size_t)nsteps * 8 * C);
  const int c = threadIdx.x % CP, pl = threadIdx.x / CP;
  const int p = blockIdx.x * NPC + pl;
  const bool act = c < C && p < d.P;
  const int cc = c < C ? c : 0, pc = p < d.P ? p : 0;
  const double wcd = g.catw[cc];
  const float4 pi4 = make_float4((float)g.pi[0], (float)g.pi[1], (float)g.pi[2], (float)g.pi[3]);
  WalkOp ring[kWalkDepth];
#pragma unroll
  for (int k = 0; k < kWalkDepth; k++) walk_fetch<false, NPC>(g, sd, codes, k, nsteps, cc, pc, pl, ring[k]);
  for (int i0 = 0; i0 < nsteps; i0 += kWalkDepth) {
#pragma unroll
    for (int k = 0; k < kWalkDepth; k++) {
      const int i = i0 + k;
      if (i < nsteps) {
        const WalkOp f = ring[k];
        walk_fetch<false, NPC>(g, sd, codes, i + kWalkDepth, nsteps, cc, pc, pl, ring[k]);
        const int4 h = sd[4 * i], q0 = sd[4 * i + 1], q1 = sd[4 * i + 2], sl = sd[4 * i + 3];
        const float4 *r0 = rows + (size_t)i * 8 * C + 4 * cc;
        const float4 *r1 = r0 + 4 * C;
        const float4 uu = h.z ? scl4(pi4, (float)(wcd * g.site_inv[pc]))
                              : vals[h.y * kWalkThr + threadIdx.x];
        const float4 s0 = walk_S(q0, f.l0, r0, nullptr);
        const float4 s1 = walk_S(q1, f.l1, r1, nullptr);
        if (q0.x != kTip) {
          const float4 U = matvec(r0, pow2_scale(mul4(uu, s1), f.e));
          if (act) g.pre[((size_t)(q0.y - d.N) * C + c) * d.P + p] = U;
          if (sl.x >= 0) vals[sl.x * kWalkThr + threadIdx.x] = U;
        }
        if (q1.x != kTip) {
          const float4 U = matvec(r1, pow2_scale(mul4(uu, s0), f.e));
          if (act) g.pre[((size_t)(q1.y - d.N) * C + c) * d.P + p] = U;
          if (sl.y >= 0) vals[sl.y * kWalkThr + threadIdx.x] = U;
        }
      }
    }
  }
}

// G[v][c][ij] = sum over the tiles of branch v, compensated FP32 (CSum),
// fixed order: the four threads of a quad take every fourth tile and combine
// by shuffles.
__global__ void k4_G_reduce(Dims d, int gstride, const int *__restrict__ parent,
                            const int *__restrict__ nt, const float *__restrict__ Gpart,
                            double *__restrict__ G) {
  pdl_wait();  // the last adjoint level's tile sums
  pdl_trigger();
  const long long t4 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long idx = t4 >> 2;
  const int part = (int)(t4 & 3);
  const bool live = idx < (long long)d.nn * d.C * 16;
  CSum acc;  // compensated FP32: FP64-class accuracy without FP64 instructions
  if (live) {
    const int ij = (int)(idx & 15);
    const int c = (int)((idx >> 4) % d.C);
    const int v = (int)(idx / (16LL * d.C));
    if (parent[v] >= 0) {
      const int n = nt[v];
      const float *src = Gpart + ((size_t)v * gstride * d.C + c) * 16 + ij;
#pragma unroll 4
      for (int t = part; t < n; t += 4) acc.add(src[(size_t)t * d.C * 16]);
    }
  }
  acc.merge(acc.shfl_xor(1));
  acc.merge(acc.shfl_xor(2));
  if (live && part == 0) G[idx] = acc.value();
}

K4Args make_args(epoch_ctx *c) {
  K4Args a{};
  a.d = c->d;
  a.PT = reinterpret_cast<const float4 *>(c->d_PT32);
  a.pairS = reinterpret_cast<const float4 *>(c->d_pairS);
  a.pairL = reinterpret_cast<const float4 *>(c->d_pairL);
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
  a.gstride = k4_tiles(c->d.P);
  a.top_begin = c->k4_top_begin;
  a.desc = c->d_k4_walk + c->k4_desc_off;
  a.pw = c->d_pw;
  a.site_lnl = c->d_site_lnl;
  a.lnl_part = c->d_lnl_part;
  a.lnl = c->d_lnl;
  a.esum = c->d_k4_esum;
  a.ctl = c->d_ctl;
  a.status = c->d_status;
  return a;
}

// largest table set of a node: two cherry children in the pre-order pass,
// plus the one-hot rows of the tip codes
size_t table_smem(const Dims &d) {
  return sizeof(float4) * (2 * d.C * (2 * d.NR * d.NR + 4) + d.NR);
}
size_t pre_smem(const Dims &d) { return table_smem(d) + sizeof(float4) * kStageF4; }

int pow2_at_least(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

size_t walk_smem(int C, int nsteps, int slots) {
  const int npc = kWalkThr / pow2_at_least(C);  // patterns per walk CTA
  return sizeof(float4) * ((size_t)nsteps * (4 + 8 * C) + (size_t)kWalkThr * slots) +
         sizeof(int) * (size_t)nsteps * 2 * npc;
}


template <int CP>
cudaError_t walk(epoch_ctx *c, bool post) {
  K4Args a = make_args(c);
  const int n = post ? c->k4_walk_post : c->k4_walk_pre;
  if (n == 0) return cudaSuccess;
  const int4 *W = c->d_k4_walk + (post ? 0 : 4 * c->k4_walk_post);
  const int slots = post ? c->k4_slots_post : c->k4_slots_pre;
  const size_t smem = walk_smem(c->d.C, n, slots);
  const int grid = ceil_div(c->d.P, kWalkThr / CP);
  if (post) {
    cudaFuncSetAttribute(k4_walk_post<CP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaError_t e = launch_pdl(k4_walk_post<CP>, dim3(grid), dim3(kWalkThr), smem, c->stream, a, W, n);
    if (e != cudaSuccess) return e;
  } else {
    cudaFuncSetAttribute(k4_walk_pre<CP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaError_t e = launch_pdl(k4_walk_pre<CP>, dim3(grid), dim3(kWalkThr), smem, c->stream, a, W, n);
    if (e != cudaSuccess) return e;
  }
  c->launches++;
  return cudaGetLastError();
}

cudaError_t walk_dispatch(epoch_ctx *c, bool post) {
  switch (pow2_at_least(c->d.C)) {
    case 1: return walk<1>(c, post);
    case 2: return walk<2>(c, post);
    case 4: return walk<4>(c, post);
    default: return walk<8>(c, post);
  }
}

// Tiles per CTA for a post-order level of w nodes and T0 fine tiles: the
// fewest rounds of resident CTAs (slots), a CTA's fixed cost (its descriptor
// and tables) counted as three tiles' worth.
int pick_post_m(int w, int T0, int slots) {
  int best = 1;
  long long best_cost = -1;
  for (int m = 1; m <= T0; m++) {
    const long long ctas = (long long)w * ((T0 + m - 1) / m);
    const long long cost = (ctas + slots - 1) / slots * (3 + m);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = m;
    }
  }
  return best;
}

template <int CMAX>
cudaError_t post(epoch_ctx *c) {
  K4Args a = make_args(c);
  const size_t smem = sizeof(float4) * ((size_t)post_tables_f4(c->d) + 2 * 2 * CMAX * kThr);
  cudaError_t err = cudaFuncSetAttribute(k4_post<CMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  int dev = 0, nsm = 0, per_sm = 0;
  err = cudaGetDevice(&dev);
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (err == cudaSuccess)
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k4_post<CMAX>, kThr, smem);
  if (err != cudaSuccess) return err;
  const int slots = std::max(1, nsm * per_sm), T0 = k4_tiles(c->d.P);
  const int last = std::max(c->k4_top, c->k4_first_level);
  for (int l = c->k4_first_level; l < last; l++) {
    const int w = c->h_level_off[l + 1] - c->h_level_off[l];
    const int m = pick_post_m(w, T0, slots);
    // the first level's predecessor wrote the cherry tables it loads
    const int early = l > c->k4_first_level ? 1 : 0;
    cudaError_t e = launch_pdl(k4_post<CMAX>, dim3(ceil_div(T0, m), w), dim3(kThr), smem,
                               c->stream, a, c->h_level_off[l], early, m);
    if (e != cudaSuccess) return e;
    c->launches++;
  }
  // the walk ends with the root: site sums, per-pattern lnL and the log-sum
  return walk_dispatch(c, true);
}

cudaError_t pre(epoch_ctx *c) {
  K4Args a = make_args(c);
  const size_t smem = pre_smem(c->d);
  cudaFuncSetAttribute(k4_pre, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int Cp = pow2_at_least(c->d.C);
  cudaError_t err = walk_dispatch(c, false);
  if (err != cudaSuccess) return err;
  for (size_t i = 0; i + 2 < c->h_k4_launch.size(); i += 3) {
    const int off = c->h_k4_launch[i], w = c->h_k4_launch[i + 1], m = c->h_k4_launch[i + 2];
    cudaError_t e = launch_pdl(k4_pre, dim3(ceil_div(c->d.P, kTP * m), w), dim3(kThr), smem,
                               c->stream, a, off, Cp, m);
    if (e != cudaSuccess) return e;
    c->launches++;
  }
  const long long nG = 4LL * c->d.nn * c->d.C * 16;
  cudaError_t e = launch_pdl(k4_G_reduce, dim3(ceil_div(nG, 256)), dim3(256), 0, c->stream,
                             c->d, a.gstride, (const int *)c->d_parent, (const int *)c->d_k4_nt,
                             (const float *)c->d_Gpart, c->d_G);
  c->launches++;
  return e;
}

}  // namespace

int k4_tiles(int P) { return (P + kTP - 1) / kTP; }

// Host schedule of the K = 4 passes for the current topology.
//   * walks: the top levels [k4_top, L) whose widths are all <= kWalkWidth
//     (the root's level always), as long as both walks fit kWalkSlots value
//     slots per thread; the post-order walk starts at max(k4_top,
//     k4_first_level) because unstored cherries are read from their tables.
//   * adjoint launches, top down: levels k4_top-1 .. 0, the first of them
//     extended over the walk's nodes, whose U the walk already stored (their
//     level-order index is >= k4_top_begin, so the kernel skips the stores)
//     and for which it only forms G.  m = fine tiles per CTA, the largest of
//     4, 2, 1 that still gives >= 4 CTAs per SM.
//   * nt[v]: tiles of the launch that handled v's parent (G tile count).
void k4_schedule(epoch_ctx *c) {
  const Dims &d = c->d;
  const int N = d.N, nn = d.nn;
  const int L = (int)c->h_level_off.size() - 1;
  const std::vector<int> &off = c->h_level_off, &nodes = c->h_level_nodes, &child = c->h_child;
  std::vector<int> lvl(nn, -1);
  for (int l = 0; l < L; l++)
    for (int i = off[l]; i < off[l + 1]; i++) lvl[nodes[i]] = l;
  auto kind_of = [&](int x) {
    if (x < N) return (int)kTip;
    const int a = child[2 * (x - N)], b = child[2 * (x - N) + 1];
    return (a < N && b < N && x != c->root) ? (int)kCherry : (int)kStored;
  };
  auto kid_desc = [&](int x) {
    int4 q{kind_of(x), x, -1, -1};
    if (q.x == kCherry) {
      q.z = child[2 * (x - N)];
      q.w = child[2 * (x - N) + 1];
    }
    return q;
  };
  int top = L - 1;
  while (top > 0 && off[top] - off[top - 1] <= kWalkWidth) top--;
  std::vector<int4> post_steps, pre_steps;
  int slots_post = 0, slots_pre = 0;
  for (;; top++) {
    post_steps.clear();
    pre_steps.clear();
    const int pfirst = std::max(top, c->k4_first_level);
    // post-order walk: level-ascending; a value lives until its parent's step
    std::vector<int> slot_of(nn, -1), free_slots;
    int nslot = 0;
    for (int i = off[pfirst]; i < off[L]; i++) {
      const int u = nodes[i];
      const int x0 = child[2 * (u - N)], x1 = child[2 * (u - N) + 1];
      int4 sl{-1, -1, 0, 0};
      if (x0 >= N && lvl[x0] >= pfirst && kind_of(x0) == kStored) sl.x = slot_of[x0];
      if (x1 >= N && lvl[x1] >= pfirst && kind_of(x1) == kStored) sl.y = slot_of[x1];
      if (sl.x >= 0) free_slots.push_back(sl.x);
      if (sl.y >= 0) free_slots.push_back(sl.y);
      int out = -1;
      if (u != c->root) {
        if (!free_slots.empty()) {
          out = free_slots.back();
          free_slots.pop_back();
        } else {
          out = nslot++;
        }
        slot_of[u] = out;
      }
      post_steps.push_back(int4{u, out, u == c->root ? 1 : 0, 0});
      post_steps.push_back(kid_desc(x0));
      post_steps.push_back(kid_desc(x1));
      post_steps.push_back(sl);
    }
    slots_post = nslot;
    // pre-order walk: level-descending; a U lives from its parent's step to
    // its own
    std::fill(slot_of.begin(), slot_of.end(), -1);
    free_slots.clear();
    nslot = 0;
    for (int l = L - 1; l >= top; l--)
      for (int i = off[l]; i < off[l + 1]; i++) {
        const int u = nodes[i];
        const int x0 = child[2 * (u - N)], x1 = child[2 * (u - N) + 1];
        if (x0 < N && x1 < N) continue;  // no U to form below u
        const int in = slot_of[u];
        if (in >= 0) free_slots.push_back(in);
        int4 sl{-1, -1, 0, 0};
        auto take = [&]() {
          if (!free_slots.empty()) {
            const int s = free_slots.back();
            free_slots.pop_back();
            return s;
          }
          return nslot++;
        };
        // a child that is itself a later step keeps its U in a slot
        if (x0 >= N && lvl[x0] >= top && kind_of(x0) == kStored) slot_of[x0] = sl.x = take();
        if (x1 >= N && lvl[x1] >= top && kind_of(x1) == kStored) slot_of[x1] = sl.y = take();
        pre_steps.push_back(int4{u, in, u == c->root ? 1 : 0, 0});
        pre_steps.push_back(kid_desc(x0));
        pre_steps.push_back(kid_desc(x1));
        pre_steps.push_back(sl);
      }
    slots_pre = nslot;
    const bool fits = slots_post <= kWalkSlots && slots_pre <= kWalkSlots &&
                      walk_smem(d.C, (int)post_steps.size() / 4, slots_post) <= kWalkSmem &&
                      walk_smem(d.C, (int)pre_steps.size() / 4, slots_pre) <= kWalkSmem;
    if (fits || top >= L - 1) break;
  }
  c->k4_top = top;
  c->k4_top_begin = off[top];
  c->k4_walk_post = (int)post_steps.size() / 4;
  c->k4_walk_pre = (int)pre_steps.size() / 4;
  c->k4_slots_post = slots_post;
  c->k4_slots_pre = slots_pre;
  c->h_k4_walk = post_steps;
  c->h_k4_walk.insert(c->h_k4_walk.end(), pre_steps.begin(), pre_steps.end());
  // level kernels: per internal node in level order {u, 0, 0, 0} and its two
  // children's descriptors, the one of smaller kind first, so that a CTA
  // learns its node and both children with one round of loads
  c->k4_desc_off = (int)c->h_k4_walk.size();
  for (int i = 0; i < off[L]; i++) {
    const int u = nodes[i];
    int4 q0 = kid_desc(child[2 * (u - N)]), q1 = kid_desc(child[2 * (u - N) + 1]);
    if (q0.x > q1.x) std::swap(q0, q1);
    c->h_k4_walk.push_back(int4{u, 0, 0, 0});
    c->h_k4_walk.push_back(q0);
    c->h_k4_walk.push_back(q1);
  }
  // adjoint launches: tiles per CTA for the fewest rounds of resident CTAs
  const int T0 = k4_tiles(d.P);
  int slots = 2 * 148;
  {
    int dev = 0, nsm = 0, per_sm = 0;
    const size_t smem = pre_smem(d);
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        cudaFuncSetAttribute(k4_pre, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
            cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k4_pre, kThr, smem) == cudaSuccess &&
        nsm * per_sm > 0)
      slots = nsm * per_sm;
    cudaGetLastError();
  }
  auto pick_m = [&](int w) { return pick_post_m(w, T0, slots); };
  c->h_k4_launch.clear();
  c->h_k4_nt.assign(nn, 0);
  auto add_launch = [&](int first, int count) {
    const int m = pick_m(count);
    c->h_k4_launch.insert(c->h_k4_launch.end(), {first, count, m});
    const int nt = (T0 + m - 1) / m;
    for (int i = first; i < first + count; i++) {
      const int u = nodes[i];
      c->h_k4_nt[child[2 * (u - N)]] = nt;
      c->h_k4_nt[child[2 * (u - N) + 1]] = nt;
    }
  };
  if (top == 0) {
    add_launch(0, off[L]);
  } else {
    add_launch(off[top - 1], off[L] - off[top - 1]);
    for (int l = top - 2; l >= 0; l--) add_launch(off[l], off[l + 1] - off[l]);
  }
}

cudaError_t launch_pair_tables_k4(epoch_ctx *c) {
  if (c->d.N < 2) return cudaSuccess;
  cudaError_t e = launch_pdl(k4_pair_tables, dim3(c->d.N - 1), dim3(128), 0, c->stream, c->d,
                             reinterpret_cast<const float4 *>(c->d_PT32),
                             (const int *)c->d_child, c->root,
                             reinterpret_cast<float4 *>(c->d_pairS),
                             reinterpret_cast<float4 *>(c->d_pairL));
  c->launches++;
  return e;
}

cudaError_t launch_partials_k4(epoch_ctx *c) {
  if (c->d.C <= 4) return post<4>(c);
  return post<8>(c);
}

cudaError_t launch_preorder_k4(epoch_ctx *c) { return pre(c); }

}  // namespace epoch
