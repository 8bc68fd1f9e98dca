// k_forest.cu -- the batched entry points (epoch_batch_*): log-likelihoods of
// many independent trees of uneven size, each with its own epochs and rate
// matrices, in ONE persistent kernel launch replayed from a CUDA graph.
//
// The method per tree is the one of the single-tree path (Eq. convolution,
// Eq. partial_likelihood, the root sum); what differs is how the branch
// matrices are applied.  The trees of this workload are large-K discrete
// traits with few patterns and general (non-reversible) Q, so instead of
// forming P = prod_k exp(dt_k Q_k) (K^3 per uniformisation term) the kernel
// applies each segment's exponential to the partial vectors directly by
// uniformisation (Jensen): with mu >= max_i |q_ii| and R = I + Q / mu
// (nonnegative, rows summing to one),
//     exp(dt Q) x = sum_m Poisson(m; mu dt) R^m x,
// truncated once a bound on the Poisson tail is below kTail (R^m never
// increases max(x), so that is also the error relative to max(x)).  A segment
// with mu dt > 30 is applied as equal pieces of mu dt <= 30, so that the first
// Poisson weight exp(-mu dt) never underflows.  Every term is nonnegative, so
// FP32 loses nothing to cancellation.  Segments are applied
// from the child end upwards (the left factor of Eq. convolution is the
// parent end).
//
// Work distribution: a CTA takes whole trees from an atomic queue ordered
// by decreasing estimated cost (longest first); inside a tree it walks the
// post-order levels, one warp per internal node, lanes over states (two per
// lane, K <= 64) and the up-to-four patterns of a state packed in a float4.
// The transposed R of every epoch of the tree sits in shared memory.  After
// each node the four pattern columns are rescaled by powers of two; the
// exponents are summed per pattern in shared memory (integers: order-free).
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "epoch.h"

struct epoch_batch;

namespace {

constexpr int kMaxPat = 4;          // patterns per tree (one float4 per state)
constexpr float kTail = 1e-9f;      // Poisson mass left out
constexpr int kMaxTerms = 4096;     // bound on uniformisation terms of one series
constexpr float kPiece = 30.f;      // longest mu dt of one series
constexpr int kMaxPieces = 1 << 16; // bound on the series of one segment
constexpr size_t kSmemCap = 200 * 1024;
constexpr int kMeta = 12;
enum { T_N, T_E, T_P, T_NODE, T_BND, T_Q, T_CODE, T_W, T_LVL, T_NLVL, T_L, T_ROOT };
enum { FS_NONFINITE = 1, FS_TERMS = 2 };

__device__ __forceinline__ float4 f4(float a) { return make_float4(a, a, a, a); }
__device__ __forceinline__ void fma4(float4 &acc, float a, float4 b) {
  acc.x = fmaf(a, b.x, acc.x);
  acc.y = fmaf(a, b.y, acc.y);
  acc.z = fmaf(a, b.z, acc.z);
  acc.w = fmaf(a, b.w, acc.w);
}
__device__ __forceinline__ float4 mul4(float4 a, float4 b) {
  return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w);
}
__device__ __forceinline__ float4 scl4(float4 a, float s) {
  return make_float4(a.x * s, a.y * s, a.z * s, a.w * s);
}
__device__ __forceinline__ float max4(float4 a) { return fmaxf(fmaxf(a.x, a.y), fmaxf(a.z, a.w)); }
__device__ __forceinline__ float warp_max(float x) {
  for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}
__device__ __forceinline__ int binary_exponent(float m) {  // m = f 2^e, f in [0.5, 1)
  int e = 0;
  if (m > 0.f) {
    e = ((__float_as_int(m) >> 23) & 255) - 126;
    if (e == -126) frexpf(m, &e);
  }
  return e;
}
__device__ __forceinline__ float pow2(int e) {  // 2^e for e in [-126, 127]
  return __int_as_float((127 + e) << 23);
}

struct ForestArgs {
  int K, T, Emax;
  const int *meta;       // [T][kMeta]
  const int *order;      // [T] trees by decreasing cost
  const double *heights; // concatenated [sum 2N_t - 1]
  const int *child;      // concatenated [sum N_t - 1][2] (local node ids)
  const int *lvl_nodes;  // concatenated internal nodes, level-ascending (local ids)
  const int *lvl_off;    // concatenated [sum L_t + 1] (relative to the tree's node list)
  const double *bnd;     // concatenated [sum E_t - 1]
  const double *Q;       // concatenated [sum E_t][K][K]
  const double *pi;      // [T][K]
  int normalise;
  const uint8_t *codes;  // concatenated [sum N_t][P_t]
  const double *w;       // concatenated [sum P_t]
  float4 *L;             // partials [sum N_t - 1][K] float4 (patterns packed)
  double *lnl;           // [T]
  int *ctl;              // [2] queue head, CTAs done
  int *status;
  // gradient launch only
  int4 *ex;              // [sum N_t - 1] rescaling exponents of every internal node
  double *dseg;          // [sum 2N_t - 1][Emax] d lnL / d (segment length), by epoch
  float4 *chain;         // per warp [2][Emax][K]: forward vectors at segment tops
  double *dh;            // [sum 2N_t - 1] d lnL / d node height
  double *db;            // [sum E_t - 1] d lnL / d boundary
  double *dbot;          // [sum 2N_t - 1] the bottom-segment term of each branch
  int2 *span;            // [sum 2N_t - 1] epochs of each branch's bottom and top segments
};

// One uniformisation series, x <- exp(dt Q_e) x with mu dt = mt in (0, kPiece]
// (TR: x <- exp(dt Q_e)^T x, the adjoint, with R^T for R): the first Poisson
// weight exp(-mt) >= exp(-kPiece) stays far above the FP32 underflow
// threshold.  buf = this warp's K float4.  RT holds R transposed, RT[j K + i]
// = R_ij.
template <bool TR>
__device__ __forceinline__ void apply_piece(const ForestArgs &g, const float *RT, float mt, int K,
                                            float4 &x0, float4 &x1, float4 *buf, int lane) {
  const bool has0 = lane < K, has1 = lane + 32 < K;
  float wgt = expf(-mt);
  float4 a0 = scl4(x0, wgt), a1 = scl4(x1, wgt);
  float4 t0 = x0, t1 = x1;
  int m = 0;
  // stop once m + 1 > mu dt and the geometric bound on the remaining Poisson
  // mass, wgt (m + 1) / (m + 1 - mu dt), is below kTail
  while (true) {
    const float r = (float)(m + 1) - mt;
    if (r > 0.f && wgt * (float)(m + 1) <= kTail * r) break;
    if (m >= kMaxTerms) {
      if (lane == 0) atomicOr(g.status, FS_TERMS);
      break;
    }
    // t <- R t (or R^T t): warp matvec through shared memory; buf holds K
    // entries, so lanes >= K neither write nor read a row
    __syncwarp();
    if (has0) buf[lane] = t0;
    if (has1) buf[lane + 32] = t1;
    __syncwarp();
    float4 n0 = f4(0.f), n1 = f4(0.f);
    for (int j = 0; j < K; j++) {
      const float4 tj = buf[j];
      if (has0) fma4(n0, TR ? RT[lane * K + j] : RT[j * K + lane], tj);
      if (has1) fma4(n1, TR ? RT[(lane + 32) * K + j] : RT[j * K + lane + 32], tj);
    }
    t0 = n0;
    t1 = n1;
    m++;
    wgt *= mt / (float)m;
    fma4(a0, wgt, t0);
    if (has1) fma4(a1, wgt, t1);
  }
  x0 = a0;
  x1 = a1;
}

// x <- exp(dt Q_e) x (TR: its transpose) for the lane's two states.  A
// segment with mu dt above kPiece is applied as n = ceil(mu dt / kPiece)
// equal pieces (exp(dt Q) = exp(dt Q / n)^n), so that no series starts from an
// underflowed weight.  A segment longer than kMaxPieces pieces (or a
// non-finite one) sets FS_TERMS.
template <bool TR = false>
__device__ __forceinline__ void apply_segment(const ForestArgs &g, const float *RT, float mu, float dt, int K,
                              float4 &x0, float4 &x1, float4 *buf, int lane) {
  const float mt = mu * dt;
  if (!(mt > 0.f)) return;  // zero length: identity
  int n = 1;
  if (mt > kPiece) {
    if (!(mt <= kPiece * (float)kMaxPieces)) {
      if (lane == 0) atomicOr(g.status, FS_TERMS);
      return;
    }
    n = (int)ceilf(mt / kPiece);
  }
  const float mp = mt / (float)n;
  for (int i = 0; i < n; i++) apply_piece<TR>(g, RT, mp, K, x0, x1, buf, lane);
}

__device__ __forceinline__ float4 warp_sum4(float4 v) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    v.z += __shfl_xor_sync(0xffffffffu, v.z, o);
    v.w += __shfl_xor_sync(0xffffffffu, v.w, o);
  }
  return v;
}

// The indicator vector of a tip's code for the lane's two states (code K =
// missing: all ones), four patterns packed.
__device__ __forceinline__ void tip_vector(const uint8_t *cv, int P, int K, int lane, float4 &x0,
                                           float4 &x1) {
  float c4[4];
#pragma unroll
  for (int p = 0; p < kMaxPat; p++) c4[p] = p < P ? (float)cv[p] : -1.f;
  auto ind = [&](int i) {
    float4 r;
    r.x = (c4[0] == (float)i || c4[0] == (float)K) ? 1.f : 0.f;
    r.y = (c4[1] == (float)i || c4[1] == (float)K) ? 1.f : 0.f;
    r.z = (c4[2] == (float)i || c4[2] == (float)K) ? 1.f : 0.f;
    r.w = (c4[3] == (float)i || c4[3] == (float)K) ? 1.f : 0.f;
    return r;
  };
  x0 = lane < K ? ind(lane) : f4(0.f);
  x1 = lane + 32 < K ? ind(lane + 32) : f4(0.f);
}

// Epochs of the bottom and top segments of the branch [hv, hu]: a segment
// belongs to the epoch of its lower end; a zero-length branch has one
// zero-length segment in the epoch of hv.
__device__ __forceinline__ void branch_epochs(const double *b, int E, double hv, double hu,
                                              int &ebot, int &etop) {
  ebot = 0;
  while (ebot < E - 1 && b[ebot] <= hv) ebot++;
  etop = 0;
  while (etop < E - 1 && b[etop] < hu) etop++;
  etop = max(etop, ebot);
}

// One CTA per tree at a time.  GRAD = false: post-order pruning and the root
// log-sum.  GRAD = true: then the pre-order adjoint of the same tree in the
// same CTA, and d lnL / d (node heights, boundaries).
//
// Adjoint (per pattern; tilde = stored, rescaled values): L~_u = S~_v o S~_w
// 2^-e_u with S~_x = P_x L~_x; U~_root = pi / s~ (s~ = pi . L~_root), and for
// a child v of u, X~_v = U~_u o S~_w 2^-e_u = d log site / d S~_v, U~_v =
// P_v^T X~_v.  For the segments of branch v, z_k at the top of segment k
// (z_0 = S~_v) and zb_k the adjoint there (zb_0 = X~_v), the derivative of
// log site by the segment's length is zb_k . Q_e z_k = mu_e zb_k . (R_e z_k -
// z_k) (Eq. convolution differentiated; exp(t Q) commutes with Q), and zb
// moves down a segment by exp(dt Q_e)^T.  U~ overwrites L~ in place: a
// node's L~ is last read when its parent forms its branch.
template <bool GRAD>
__global__ void __launch_bounds__(256, 2) k_forest(ForestArgs g) {
  extern __shared__ float smem[];
  __shared__ int s_tree;
  __shared__ int s_exp[kMaxPat];
  __shared__ double s_b[64];
  __shared__ float s_mu[64];
  const int K = g.K, KK = K * K;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  float *RT = smem;                                          // [Emax][K][K] transposed R
  float4 *wbuf = reinterpret_cast<float4 *>(RT + (size_t)g.Emax * KK);  // [nwarps][K]
  float4 *buf = wbuf + (size_t)warp * K;
  // this warp's forward vectors at the segment tops of both children
  float4 *chain = GRAD ? g.chain + ((size_t)blockIdx.x * nwarps + warp) * 2 * g.Emax * K : nullptr;
  while (true) {
    if (threadIdx.x == 0) s_tree = atomicAdd(&g.ctl[0], 1);
    __syncthreads();
    const int it = s_tree;
    if (it >= g.T) break;
    const int t = g.order[it];
    const int *mt = g.meta + (size_t)t * kMeta;
    const int N = mt[T_N], E = mt[T_E], P = mt[T_P];
    const double *hgt = g.heights + mt[T_NODE];
    const int *child = g.child + 2 * (size_t)mt[T_L];  // [N-1][2] of this tree
    const uint8_t *codes = g.codes + mt[T_CODE];
    float4 *Lt = g.L + (size_t)mt[T_L] * K;
    // rate matrices of the tree: normalise, mu, transposed R (FP64 -> FP32)
    for (int e = warp; e < E; e += nwarps) {
      const double *q = g.Q + (size_t)(mt[T_Q] + e) * KK;
      const double *pi = g.pi + (size_t)t * K;
      double cs = 0.0, mx = 0.0;
      for (int i = lane; i < K; i += 32) {
        cs -= pi[i] * q[i * K + i];
        mx = fmax(mx, -q[i * K + i]);
      }
      for (int o = 16; o > 0; o >>= 1) {
        cs += __shfl_xor_sync(0xffffffffu, cs, o);
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      }
      const double c = (g.normalise && cs > 0.0) ? cs : 1.0;
      const double mu = mx / c;
      if (lane == 0) s_mu[e] = (float)mu;
      const double inv = mu > 0.0 ? 1.0 / (c * mu) : 0.0;
      float *R = RT + (size_t)e * KK;
      for (int idx = lane; idx < KK; idx += 32) {
        const int i = idx / K, j = idx % K;  // R[i][j] stored at [j][i]
        R[j * K + i] = (float)((i == j ? 1.0 : 0.0) + q[idx] * inv);
      }
    }
    for (int j = threadIdx.x; j < E - 1; j += blockDim.x) s_b[j] = g.bnd[mt[T_BND] + j];
    if (threadIdx.x < kMaxPat) s_exp[threadIdx.x] = 0;
    __syncthreads();
    const int *lvl = g.lvl_nodes + mt[T_L];  // the tree's N-1 internal nodes
    const int *loff = g.lvl_off + mt[T_LVL];
    const int nl = mt[T_NLVL], root = mt[T_ROOT];
    for (int l = 0; l < nl; l++) {
      for (int k = loff[l] + warp; k < loff[l + 1]; k += nwarps) {
        const int u = lvl[k];
        float4 s0[2], s1[2];
#pragma unroll
        for (int side = 0; side < 2; side++) {
          const int v = child[2 * (u - N) + side];
          float4 x0, x1;
          if (v < N) {  // tip: indicator of the observed state (K = missing)
            tip_vector(codes + (size_t)v * P, P, K, lane, x0, x1);
          } else {
            const float4 *src = Lt + (size_t)(v - N) * K;
            x0 = lane < K ? src[lane] : f4(0.f);
            x1 = lane + 32 < K ? src[lane + 32] : f4(0.f);
          }
          // segments from the child end up (a segment belongs to the epoch
          // of its lower end; boundaries strictly increase)
          const double hv = hgt[v], hu = hgt[u];
          double lo = hv;
          int e = 0;
          while (e < E - 1 && s_b[e] <= lo) e++;
          while (lo < hu) {
            const double top = (e < E - 1 && s_b[e] < hu) ? s_b[e] : hu;
            apply_segment(g, RT + (size_t)e * KK, s_mu[e], (float)(top - lo), K, x0, x1, buf, lane);
            lo = top;
            e++;
          }
          s0[side] = x0;
          s1[side] = x1;
        }
        float4 l0 = mul4(s0[0], s0[1]), l1 = mul4(s1[0], s1[1]);
        // per-pattern power-of-two rescaling
        float mx = fmaxf(l0.x, l1.x), my = fmaxf(l0.y, l1.y), mz = fmaxf(l0.z, l1.z),
              mw = fmaxf(l0.w, l1.w);
        mx = warp_max(mx);
        my = warp_max(my);
        mz = warp_max(mz);
        mw = warp_max(mw);
        if (!(fmaxf(fmaxf(mx, my), fmaxf(mz, mw)) <= 3.0e38f) && lane == 0)
          atomicOr(g.status, FS_NONFINITE);
        const int ex = binary_exponent(mx), ey = binary_exponent(my), ez = binary_exponent(mz),
                  ew = binary_exponent(mw);
        const int es[4] = {max(ex, -126), max(ey, -126), max(ez, -126), max(ew, -126)};
        const float4 sc = make_float4(pow2(-es[0]), pow2(-es[1]), pow2(-es[2]), pow2(-es[3]));
        l0 = mul4(l0, sc);
        l1 = mul4(l1, sc);
        float4 *dst = Lt + (size_t)(u - N) * K;
        if (lane < K) dst[lane] = l0;
        if (lane + 32 < K) dst[lane + 32] = l1;
        if (lane == 0) {
#pragma unroll
          for (int p = 0; p < kMaxPat; p++)
            if (p < P) atomicAdd(&s_exp[p], es[p]);
          if (GRAD) g.ex[mt[T_L] + (u - N)] = make_int4(es[0], es[1], es[2], es[3]);
        }
      }
      __syncthreads();
    }
    // root: lnL = sum_p w_p (log sum_i pi_i L_root(i,p) + ln2 * sum_u e_u(p))
    if (warp == 0) {
      float4 *Lr = Lt + (size_t)(root - N) * K;
      const double *pi = g.pi + (size_t)t * K;
      double sp[4] = {0.0, 0.0, 0.0, 0.0};
      for (int i = lane; i < K; i += 32) {
        const float4 v = Lr[i];
        sp[0] += pi[i] * (double)v.x;
        sp[1] += pi[i] * (double)v.y;
        sp[2] += pi[i] * (double)v.z;
        sp[3] += pi[i] * (double)v.w;
      }
      for (int p = 0; p < 4; p++)
        for (int o = 16; o > 0; o >>= 1) sp[p] += __shfl_xor_sync(0xffffffffu, sp[p], o);
      if (lane == 0) {
        double acc = 0.0;
#pragma unroll
        for (int p = 0; p < kMaxPat; p++) {
          const double wp = p < P ? g.w[mt[T_W] + p] : 0.0;
          if (wp != 0.0) acc += wp * (log(sp[p]) + 0.69314718055994530942 * (double)s_exp[p]);
        }
        g.lnl[t] = acc;
      }
      if (GRAD) {
        // U~_root = pi / s~ per pattern (0 for an impossible or absent
        // pattern: it adds nothing to the gradient), over L~_root
        float inv[4];
#pragma unroll
        for (int p = 0; p < kMaxPat; p++) inv[p] = (p < P && sp[p] > 0.0) ? (float)(1.0 / sp[p]) : 0.f;
        for (int i = lane; i < K; i += 32) {
          const float pf = (float)pi[i];
          Lr[i] = make_float4(pf * inv[0], pf * inv[1], pf * inv[2], pf * inv[3]);
        }
      }
    }
    __syncthreads();
    if (GRAD) {
      const double *w = g.w + mt[T_W];
      double *dseg = g.dseg + (size_t)mt[T_NODE] * g.Emax;
      // pre-order, top level first: a warp per node forms both children's
      // branches
      for (int l = nl - 1; l >= 0; l--) {
        for (int k = loff[l] + warp; k < loff[l + 1]; k += nwarps) {
          const int u = lvl[k];
          float4 *Uu = Lt + (size_t)(u - N) * K;
          const float4 uu0 = lane < K ? Uu[lane] : f4(0.f);
          const float4 uu1 = lane + 32 < K ? Uu[lane + 32] : f4(0.f);
          const int4 eu = g.ex[mt[T_L] + (u - N)];
          const float4 su = make_float4(pow2(-eu.x), pow2(-eu.y), pow2(-eu.z), pow2(-eu.w));
          float4 top0[2], top1[2];
          int eb[2], et[2];
          // forward: each child's vectors at its segment tops, by epoch
#pragma unroll
          for (int side = 0; side < 2; side++) {
            const int v = child[2 * (u - N) + side];
            float4 x0, x1;
            if (v < N) {
              tip_vector(codes + (size_t)v * P, P, K, lane, x0, x1);
            } else {
              const float4 *src = Lt + (size_t)(v - N) * K;
              x0 = lane < K ? src[lane] : f4(0.f);
              x1 = lane + 32 < K ? src[lane + 32] : f4(0.f);
            }
            const double hv = hgt[v], hu = hgt[u];
            branch_epochs(s_b, E, hv, hu, eb[side], et[side]);
            float4 *ch = chain + (size_t)side * g.Emax * K;
            if (hv >= hu) {  // zero length: one segment, P = I
              if (lane < K) ch[eb[side] * K + lane] = x0;
              if (lane + 32 < K) ch[eb[side] * K + lane + 32] = x1;
            }
            double lo = hv;
            int e = eb[side];
            while (lo < hu) {
              const double top = (e < E - 1 && s_b[e] < hu) ? s_b[e] : hu;
              apply_segment(g, RT + (size_t)e * KK, s_mu[e], (float)(top - lo), K, x0, x1, buf, lane);
              if (lane < K) ch[e * K + lane] = x0;
              if (lane + 32 < K) ch[e * K + lane + 32] = x1;
              lo = top;
              e++;
            }
            top0[side] = x0;  // S~ of this child
            top1[side] = x1;
          }
          // adjoint: each child's branch from its top down
          double dtop = 0.0;  // lane 0: the top-segment terms of both branches
#pragma unroll
          for (int side = 0; side < 2; side++) {
            const int v = child[2 * (u - N) + side];
            const int o = 1 - side;
            float4 zb0 = mul4(mul4(uu0, top0[o]), su);  // X~_v
            float4 zb1 = mul4(mul4(uu1, top1[o]), su);
            const float4 *ch = chain + (size_t)side * g.Emax * K;
            double *drow = dseg + (size_t)v * g.Emax;
            const double hv = hgt[v], hu = hgt[u];
            for (int e = et[side]; e >= eb[side]; e--) {
              // mu_e zb . (R_e z - z), z the forward vector at the segment top
              const float4 z0 = lane < K ? ch[e * K + lane] : f4(0.f);
              const float4 z1 = lane + 32 < K ? ch[e * K + lane + 32] : f4(0.f);
              const float *R = RT + (size_t)e * KK;
              __syncwarp();
              if (lane < K) buf[lane] = z0;
              if (lane + 32 < K) buf[lane + 32] = z1;
              __syncwarp();
              float4 r0 = f4(0.f), r1 = f4(0.f);
              for (int j = 0; j < K; j++) {
                const float4 zj = buf[j];
                if (lane < K) fma4(r0, R[j * K + lane], zj);
                if (lane + 32 < K) fma4(r1, R[j * K + lane + 32], zj);
              }
              float4 d = mul4(zb0, make_float4(r0.x - z0.x, r0.y - z0.y, r0.z - z0.z, r0.w - z0.w));
              const float4 d1 = mul4(zb1, make_float4(r1.x - z1.x, r1.y - z1.y, r1.z - z1.z, r1.w - z1.w));
              d = make_float4(d.x + d1.x, d.y + d1.y, d.z + d1.z, d.w + d1.w);
              d = warp_sum4(d);
              if (lane == 0) {
                const double ds = (P > 0 ? w[0] * (double)d.x : 0.0) + (P > 1 ? w[1] * (double)d.y : 0.0) +
                                  (P > 2 ? w[2] * (double)d.z : 0.0) + (P > 3 ? w[3] * (double)d.w : 0.0);
                drow[e] = (double)s_mu[e] * ds;
              }
              // zb down this segment
              const double lo = (e > eb[side]) ? s_b[e - 1] : hv;
              const double top = (e < et[side]) ? s_b[e] : hu;
              if (top > lo)
                apply_segment<true>(g, R, s_mu[e], (float)(top - lo), K, zb0, zb1, buf, lane);
            }
            if (lane == 0) {
              for (int e = 0; e < g.Emax; e++)
                if (e < eb[side] || e > et[side] || e >= E) drow[e] = 0.0;
              dtop += drow[et[side]];
              g.dbot[mt[T_NODE] + v] = drow[eb[side]];
              g.span[mt[T_NODE] + v] = make_int2(eb[side], et[side]);
            }
            if (v >= N) {  // U~_v over L~_v
              float4 *dst = Lt + (size_t)(v - N) * K;
              if (lane < K) dst[lane] = zb0;
              if (lane + 32 < K) dst[lane + 32] = zb1;
            }
          }
          if (lane == 0) g.dh[mt[T_NODE] + u] = dtop;
        }
        __syncthreads();
      }
      // d lnL / d h_x: the top-segment terms of x's child branches (written by
      // x's warp) minus the bottom-segment term of x's own branch (written by
      // its parent's); d lnL / d b_j: over the branches that cross b_j, the
      // term of the segment below minus the one above.  Fixed order, no
      // atomics.
      const int nn = 2 * N - 1;
      double *dh = g.dh + mt[T_NODE];
      const double *dbot = g.dbot + mt[T_NODE];
      const int2 *span = g.span + mt[T_NODE];
      for (int x = threadIdx.x; x < nn; x += blockDim.x)
        dh[x] = (x >= N ? dh[x] : 0.0) - (x != root ? dbot[x] : 0.0);
      for (int j = warp; j < E - 1; j += nwarps) {
        double acc = 0.0;
        for (int x = lane; x < nn; x += 32) {
          if (x == root) continue;
          const int2 sp = span[x];
          if (sp.x <= j && j < sp.y) acc += dseg[(size_t)x * g.Emax + j] - dseg[(size_t)x * g.Emax + j + 1];
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) g.db[mt[T_BND] + j] = acc;
      }
      __syncthreads();
    }
  }
  // the last CTA to finish resets the queue for the next launch
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&g.ctl[1], 1) == (int)gridDim.x - 1) {
      g.ctl[0] = 0;
      g.ctl[1] = 0;
      __threadfence();
    }
  }
}

}  // namespace

// ===========================================================================
// host side
// ===========================================================================
struct epoch_batch {
  int K = 0, T = 0, Emax = 1;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  unsigned have = 0;  // 1 models, 2 trees, 4 tips
  int normalise = 1;
  std::vector<int> N, E, P;
  std::vector<int> meta;  // [T][kMeta]
  long long total_nodes = 0, total_internal = 0, total_bnd = 0, total_q = 0, total_codes = 0,
            total_w = 0;
  std::vector<int> lvl_off, lvl_nodes, child;
  std::vector<int> order;
  // device
  int *d_meta = nullptr, *d_order = nullptr, *d_child = nullptr, *d_lvl_nodes = nullptr,
      *d_lvl_off = nullptr, *d_ctl = nullptr, *d_status = nullptr;
  double *d_heights = nullptr, *d_bnd = nullptr, *d_Q = nullptr, *d_pi = nullptr, *d_w = nullptr,
         *d_lnl = nullptr;
  uint8_t *d_codes = nullptr;
  float4 *d_L = nullptr;
  int *h_status = nullptr;
  // launch shape (autotuned on first evaluation) and graph
  int warps = 0, ctas_per_sm = 0, n_sm = 0;
  cudaGraphExec_t graph = nullptr;
  // the gradient launch: its buffers (allocated on first use), shape, graph
  int4 *d_ex = nullptr;
  double *d_dseg = nullptr, *d_dh = nullptr, *d_db = nullptr, *d_dbot = nullptr;
  int2 *d_span = nullptr;
  float4 *d_chain = nullptr;
  int gwarps = 0, gctas_per_sm = 0;
  cudaGraphExec_t ggraph = nullptr;
  bool grad_valid = false;  // the last evaluation was a gradient evaluation
};

namespace {

epoch_status bfail(epoch_batch *b, epoch_status s, const std::string &m) {
  if (b) b->err = m;
  return s;
}
#define BCK(call, what)                                                               \
  do {                                                                                \
    cudaError_t _e = (call);                                                          \
    if (_e != cudaSuccess) return bfail(b, EPOCH_ERR_CUDA, std::string(what) + ": " + \
                                                             cudaGetErrorString(_e)); \
  } while (0)

size_t forest_smem(const epoch_batch *b, int warps) {
  return sizeof(float) * (size_t)b->Emax * b->K * b->K + sizeof(float4) * (size_t)warps * b->K;
}

ForestArgs forest_args(epoch_batch *b) {
  ForestArgs a{};
  a.K = b->K;
  a.T = b->T;
  a.Emax = b->Emax;
  a.meta = b->d_meta;
  a.order = b->d_order;
  a.heights = b->d_heights;
  a.child = b->d_child;
  a.lvl_nodes = b->d_lvl_nodes;
  a.lvl_off = b->d_lvl_off;
  a.bnd = b->d_bnd;
  a.Q = b->d_Q;
  a.pi = b->d_pi;
  a.normalise = b->normalise;
  a.codes = b->d_codes;
  a.w = b->d_w;
  a.L = b->d_L;
  a.lnl = b->d_lnl;
  a.ctl = b->d_ctl;
  a.status = b->d_status;
  a.ex = b->d_ex;
  a.dseg = b->d_dseg;
  a.chain = b->d_chain;
  a.dh = b->d_dh;
  a.db = b->d_db;
  a.dbot = b->d_dbot;
  a.span = b->d_span;
  return a;
}

constexpr int kMaxCtasPerSm = 3;
constexpr int kMaxWarps = 8;

template <bool GRAD>
cudaError_t forest_launch(epoch_batch *b, int warps, int ctas_per_sm) {
  const size_t smem = forest_smem(b, warps);
  cudaError_t e = cudaFuncSetAttribute(k_forest<GRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = std::max(1, std::min(b->T, b->n_sm * ctas_per_sm));
  k_forest<GRAD><<<grid, 32 * warps, smem, b->stream>>>(forest_args(b));
  return cudaGetLastError();
}

// Autotuner: time every launch shape that fits (warps per CTA x CTAs per SM)
// on the current inputs and keep the fastest.
template <bool GRAD>
epoch_status forest_tune(epoch_batch *b, int &best_w, int &best_c) {
  const int cand_w[] = {4, kMaxWarps};
  const int cand_c[] = {1, 2, kMaxCtasPerSm};
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0), "cudaEventCreate");
  BCK(cudaEventCreate(&e1), "cudaEventCreate");
  float best = 1e30f;
  int bw = kMaxWarps, bc = 1;
  for (int w : cand_w)
    for (int cps : cand_c) {
      const size_t smem = forest_smem(b, w);
      if (smem * cps > kSmemCap) continue;
      int nb = 0;
      if (cudaFuncSetAttribute(k_forest<GRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_forest<GRAD>, 32 * w, smem) !=
              cudaSuccess ||
          nb < cps)
        continue;
      BCK(forest_launch<GRAD>(b, w, cps), "forest launch");  // warm-up
      BCK(cudaEventRecord(e0, b->stream), "cudaEventRecord");
      for (int r = 0; r < 2; r++) BCK(forest_launch<GRAD>(b, w, cps), "forest launch");
      BCK(cudaEventRecord(e1, b->stream), "cudaEventRecord");
      BCK(cudaEventSynchronize(e1), "cudaEventSynchronize");
      float ms = 0.f;
      BCK(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
      if (ms < best) {
        best = ms;
        bw = w;
        bc = cps;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  best_w = bw;
  best_c = bc;
  return EPOCH_OK;
}

template <typename T>
cudaError_t balloc(T **p, size_t n) {
  *p = nullptr;
  return cudaMalloc((void **)p, std::max<size_t>(n, 1) * sizeof(T));
}

void invalidate(epoch_batch *b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  if (b->ggraph) cudaGraphExecDestroy(b->ggraph);
  b->ggraph = nullptr;
}

// Capture the launch of the given shape in a graph (once) and replay it.
template <bool GRAD>
epoch_status forest_replay(epoch_batch *b, cudaGraphExec_t &graph, int warps, int ctas) {
  if (!graph) {
    cudaGraph_t g = nullptr;
    BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed), "cudaStreamBeginCapture");
    cudaError_t e = forest_launch<GRAD>(b, warps, ctas);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return bfail(b, EPOCH_ERR_CUDA, "capturing the forest launch failed");
    }
    e = cudaGraphInstantiate(&graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(b, EPOCH_ERR_CUDA, cudaGetErrorString(e));
  }
  BCK(cudaGraphLaunch(graph, b->stream), "cudaGraphLaunch");
  return EPOCH_OK;
}

}  // namespace

extern "C" {

epoch_status epoch_batch_create(epoch_batch **out, int states, int n_trees, const int *n_taxa,
                                const int *n_epochs, const int *n_patterns, void *cuda_stream) {
  if (!out) return EPOCH_ERR_ARG;
  *out = nullptr;
  if (states < 2 || states > EPOCH_MAX_STATES || n_trees < 1 || !n_taxa || !n_epochs ||
      !n_patterns)
    return EPOCH_ERR_ARG;
  for (int t = 0; t < n_trees; t++)
    if (n_taxa[t] < 2 || n_epochs[t] < 1 || n_epochs[t] > EPOCH_MAX_EPOCHS || n_patterns[t] < 1 ||
        n_patterns[t] > kMaxPat)
      return EPOCH_ERR_ARG;
  epoch_batch *b = new (std::nothrow) epoch_batch();
  if (!b) return EPOCH_ERR_CAPACITY;
  b->K = states;
  b->T = n_trees;
  b->N.assign(n_taxa, n_taxa + n_trees);
  b->E.assign(n_epochs, n_epochs + n_trees);
  b->P.assign(n_patterns, n_patterns + n_trees);
  b->Emax = *std::max_element(b->E.begin(), b->E.end());
  if (forest_smem(b, 4) > kSmemCap) {
    delete b;
    return EPOCH_ERR_CAPACITY;  // the epochs' R matrices do not fit in shared memory
  }
  b->meta.assign((size_t)n_trees * kMeta, 0);
  long long nodes = 0, internal = 0, bnd = 0, q = 0, codes = 0, w = 0;
  for (int t = 0; t < n_trees; t++) {
    int *m = &b->meta[(size_t)t * kMeta];
    m[T_N] = b->N[t];
    m[T_E] = b->E[t];
    m[T_P] = b->P[t];
    m[T_NODE] = (int)nodes;
    m[T_BND] = (int)bnd;
    m[T_Q] = (int)q;
    m[T_CODE] = (int)codes;
    m[T_W] = (int)w;
    m[T_L] = (int)internal;
    nodes += 2LL * b->N[t] - 1;
    internal += b->N[t] - 1;
    bnd += b->E[t] - 1;
    q += b->E[t];
    codes += (long long)b->N[t] * b->P[t];
    w += b->P[t];
  }
  if (nodes > (1LL << 30) || codes > (1LL << 31) - 1) {
    delete b;
    return EPOCH_ERR_CAPACITY;
  }
  b->total_nodes = nodes;
  b->total_internal = internal;
  b->total_bnd = bnd;
  b->total_q = q;
  b->total_codes = codes;
  b->total_w = w;
  epoch_status s = EPOCH_OK;
  auto A = [&](cudaError_t e) {
    if (e != cudaSuccess && s == EPOCH_OK) s = bfail(b, EPOCH_ERR_CUDA, cudaGetErrorString(e));
  };
  if (cuda_stream) {
    b->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    A(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    b->own_stream = true;
  }
  int dev = 0;
  A(cudaGetDevice(&dev));
  A(cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, dev));
  const int K = states;
  A(balloc(&b->d_meta, b->meta.size()));
  A(balloc(&b->d_order, n_trees));
  A(balloc(&b->d_heights, nodes));
  A(balloc(&b->d_child, 2 * internal));
  A(balloc(&b->d_lvl_nodes, internal));
  A(balloc(&b->d_lvl_off, internal + n_trees));
  A(balloc(&b->d_bnd, bnd));
  A(balloc(&b->d_Q, q * K * K));
  A(balloc(&b->d_pi, (size_t)n_trees * K));
  A(balloc(&b->d_codes, codes));
  A(balloc(&b->d_w, w));
  A(balloc(&b->d_L, internal * K));
  A(balloc(&b->d_lnl, n_trees));
  A(balloc(&b->d_ctl, 2));
  A(balloc(&b->d_status, 1));
  A(cudaMallocHost((void **)&b->h_status, sizeof(int)));
  if (s == EPOCH_OK) {
    A(cudaMemsetAsync(b->d_ctl, 0, 2 * sizeof(int), b->stream));
    A(cudaMemsetAsync(b->d_status, 0, sizeof(int), b->stream));
  }
  if (s != EPOCH_OK) {
    epoch_batch_destroy(b);
    return s;
  }
  *out = b;
  return EPOCH_OK;
}

void epoch_batch_destroy(epoch_batch *b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  invalidate(b);
  void *bufs[] = {b->d_meta, b->d_order, b->d_heights, b->d_child, b->d_lvl_nodes, b->d_lvl_off,
                  b->d_bnd,  b->d_Q,     b->d_pi,      b->d_codes, b->d_w,         b->d_L,
                  b->d_lnl,  b->d_ctl,   b->d_status,  b->d_ex,    b->d_dseg,      b->d_chain,
                  b->d_dh,   b->d_db,    b->d_dbot,    b->d_span};
  for (void *p : bufs)
    if (p) cudaFree(p);
  if (b->h_status) cudaFreeHost(b->h_status);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

const char *epoch_batch_last_error(const epoch_batch *b) { return b ? b->err.c_str() : ""; }

epoch_status epoch_batch_set_models(epoch_batch *b, const double *boundaries, const double *Q,
                                    const double *pi, int normalise) {
  if (!b) return EPOCH_ERR_ARG;
  b->grad_valid = false;
  if (!Q || !pi || (b->total_bnd > 0 && !boundaries))
    return bfail(b, EPOCH_ERR_ARG, "NULL model array");
  const int K = b->K;
  for (int t = 0; t < b->T; t++) {
    const int *m = &b->meta[(size_t)t * kMeta];
    const double *bt = boundaries ? boundaries + m[T_BND] : nullptr;
    for (int j = 0; j < b->E[t] - 1; j++) {
      if (!std::isfinite(bt[j]) || bt[j] <= 0.0 || (j > 0 && bt[j] <= bt[j - 1]))
        return bfail(b, EPOCH_ERR_ARG, "boundaries of tree " + std::to_string(t) +
                                           " must be positive, finite and increasing");
    }
    double ps = 0.0;
    for (int i = 0; i < K; i++) {
      const double p = pi[(size_t)t * K + i];
      if (!std::isfinite(p) || p < 0.0) return bfail(b, EPOCH_ERR_NUMERIC, "bad pi");
      ps += p;
    }
    if (fabs(ps - 1.0) > 1e-9) return bfail(b, EPOCH_ERR_NUMERIC, "pi must sum to 1");
    for (int e = 0; e < b->E[t]; e++) {
      const double *q = Q + (size_t)(m[T_Q] + e) * K * K;
      for (int i = 0; i < K; i++) {
        double rs = 0.0;
        for (int j = 0; j < K; j++) {
          const double x = q[i * K + j];
          if (!std::isfinite(x) || (i != j && x < 0.0))
            return bfail(b, EPOCH_ERR_NUMERIC, "Q must be finite with nonnegative off-diagonals");
          rs += x;
        }
        if (fabs(rs) > 1e-8 * (1.0 + fabs(q[i * K + i])))
          return bfail(b, EPOCH_ERR_NUMERIC, "rows of Q must sum to zero");
      }
    }
  }
  b->normalise = normalise ? 1 : 0;
  if (b->total_bnd > 0)
    BCK(cudaMemcpyAsync(b->d_bnd, boundaries, sizeof(double) * b->total_bnd, cudaMemcpyHostToDevice,
                        b->stream),
        "cudaMemcpyAsync(boundaries)");
  BCK(cudaMemcpyAsync(b->d_Q, Q, sizeof(double) * b->total_q * K * K, cudaMemcpyHostToDevice,
                      b->stream),
      "cudaMemcpyAsync(Q)");
  BCK(cudaMemcpyAsync(b->d_pi, pi, sizeof(double) * b->T * K, cudaMemcpyHostToDevice, b->stream),
      "cudaMemcpyAsync(pi)");
  BCK(cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");  // host arrays may go away
  b->have |= 1u;
  return EPOCH_OK;
}

epoch_status epoch_batch_set_trees(epoch_batch *b, const double *heights, const int *parent) {
  if (!b) return EPOCH_ERR_ARG;
  b->grad_valid = false;
  if (!heights || !parent) return bfail(b, EPOCH_ERR_ARG, "NULL tree array");
  std::vector<int> child((size_t)2 * b->total_internal), lvl_nodes(b->total_internal), lvl_off;
  std::vector<double> cost(b->T);
  for (int t = 0; t < b->T; t++) {
    int *m = &b->meta[(size_t)t * kMeta];
    const int N = b->N[t], nn = 2 * N - 1;
    const double *h = heights + m[T_NODE];
    const int *par = parent + m[T_NODE];
    std::vector<int> cnt(nn, 0), lvl(nn, 0);
    int root = -1;
    for (int v = 0; v < nn; v++) {
      if (!std::isfinite(h[v])) return bfail(b, EPOCH_ERR_ARG, "non-finite height");
      const int u = par[v];
      if (u < 0) {
        if (root >= 0 || v < N) return bfail(b, EPOCH_ERR_ARG, "tree needs one internal root");
        root = v;
        continue;
      }
      if (u < N || u >= nn) return bfail(b, EPOCH_ERR_ARG, "parent must be an internal node");
      if (h[u] < h[v]) return bfail(b, EPOCH_ERR_ARG, "parent below child");
      if (cnt[u] >= 2) return bfail(b, EPOCH_ERR_ARG, "node with more than two children");
      child[(size_t)2 * (m[T_L] + u - N) + cnt[u]++] = v;
    }
    if (root < 0) return bfail(b, EPOCH_ERR_ARG, "no root");
    for (int u = N; u < nn; u++)
      if (cnt[u] != 2) return bfail(b, EPOCH_ERR_ARG, "internal node without two children");
    // levels: tips 0, internal 1 + max of children (iterative post-order)
    std::vector<int> st{root}, done(nn, 0);
    while (!st.empty()) {
      const int u = st.back();
      if (u < N) {
        st.pop_back();
        continue;
      }
      const int a = child[(size_t)2 * (m[T_L] + u - N)], c2 = child[(size_t)2 * (m[T_L] + u - N) + 1];
      if (!done[u]) {
        done[u] = 1;
        st.push_back(a);
        st.push_back(c2);
        if ((int)st.size() > 4 * nn) return bfail(b, EPOCH_ERR_ARG, "not a tree");
      } else {
        lvl[u] = 1 + std::max(lvl[a], lvl[c2]);
        st.pop_back();
      }
    }
    const int L = lvl[root];
    std::vector<int> count(L + 2, 0);
    for (int u = N; u < nn; u++) {
      if (!done[u]) return bfail(b, EPOCH_ERR_ARG, "node not reachable from the root");
      count[lvl[u]]++;
    }
    m[T_LVL] = (int)lvl_off.size();
    m[T_NLVL] = L;
    m[T_ROOT] = root;
    std::vector<int> start(L + 2, 0);
    for (int l = 1; l <= L; l++) start[l + 1] = start[l] + count[l];
    for (int l = 1; l <= L + 1; l++) lvl_off.push_back(start[l]);
    std::vector<int> fill(start.begin(), start.end());
    for (int u = N; u < nn; u++) lvl_nodes[(size_t)m[T_L] + fill[lvl[u]]++] = u;
    cost[t] = (double)N * b->P[t] * (1.0 + b->E[t]);
  }
  std::vector<int> order(b->T);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  b->child = child;
  b->lvl_nodes = lvl_nodes;
  b->lvl_off = lvl_off;
  b->order = order;
  invalidate(b);
  if (b->d_lvl_off) cudaFree(b->d_lvl_off);
  BCK(balloc(&b->d_lvl_off, lvl_off.size()), "cudaMalloc(levels)");
  BCK(cudaMemcpyAsync(b->d_meta, b->meta.data(), sizeof(int) * b->meta.size(),
                      cudaMemcpyHostToDevice, b->stream),
      "cudaMemcpyAsync(meta)");
  BCK(cudaMemcpyAsync(b->d_order, b->order.data(), sizeof(int) * b->T, cudaMemcpyHostToDevice,
                      b->stream),
      "cudaMemcpyAsync(order)");
  BCK(cudaMemcpyAsync(b->d_heights, heights, sizeof(double) * b->total_nodes,
                      cudaMemcpyHostToDevice, b->stream),
      "cudaMemcpyAsync(heights)");
  BCK(cudaMemcpyAsync(b->d_child, b->child.data(), sizeof(int) * b->child.size(),
                      cudaMemcpyHostToDevice, b->stream),
      "cudaMemcpyAsync(children)");
  BCK(cudaMemcpyAsync(b->d_lvl_nodes, b->lvl_nodes.data(), sizeof(int) * b->lvl_nodes.size(),
                      cudaMemcpyHostToDevice, b->stream),
      "cudaMemcpyAsync(level nodes)");
  BCK(cudaMemcpyAsync(b->d_lvl_off, b->lvl_off.data(), sizeof(int) * b->lvl_off.size(),
                      cudaMemcpyHostToDevice, b->stream),
      "cudaMemcpyAsync(level offsets)");
  BCK(cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
  b->have |= 2u;
  return EPOCH_OK;
}

epoch_status epoch_batch_set_tip_data(epoch_batch *b, const int *codes, const double *weights) {
  if (!b) return EPOCH_ERR_ARG;
  b->grad_valid = false;
  if (!codes || !weights) return bfail(b, EPOCH_ERR_ARG, "NULL tip array");
  std::vector<uint8_t> c8(b->total_codes);
  unsigned bad = 0;
  for (long long i = 0; i < b->total_codes; i++) {
    const unsigned c = (unsigned)codes[i];
    bad |= (unsigned)(c > (unsigned)b->K);
    c8[i] = (uint8_t)c;
  }
  if (bad) return bfail(b, EPOCH_ERR_ARG, "tip code out of range (0..K, K = missing)");
  for (long long i = 0; i < b->total_w; i++)
    if (!std::isfinite(weights[i]) || weights[i] < 0.0)
      return bfail(b, EPOCH_ERR_ARG, "bad pattern weight");
  BCK(cudaMemcpyAsync(b->d_codes, c8.data(), b->total_codes, cudaMemcpyHostToDevice, b->stream),
      "cudaMemcpyAsync(codes)");
  BCK(cudaMemcpyAsync(b->d_w, weights, sizeof(double) * b->total_w, cudaMemcpyHostToDevice,
                      b->stream),
      "cudaMemcpyAsync(weights)");
  BCK(cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
  b->have |= 4u;
  return EPOCH_OK;
}

epoch_status epoch_batch_evaluate_async(epoch_batch *b) {
  if (!b) return EPOCH_ERR_ARG;
  if ((b->have & 7u) != 7u)
    return bfail(b, EPOCH_ERR_ORDER, "set models, trees and tip data before evaluating");
  if (!b->warps) {
    epoch_status s = forest_tune<false>(b, b->warps, b->ctas_per_sm);
    if (s != EPOCH_OK) return s;
  }
  b->grad_valid = false;
  return forest_replay<false>(b, b->graph, b->warps, b->ctas_per_sm);
}

epoch_status epoch_batch_evaluate_gradient_async(epoch_batch *b) {
  if (!b) return EPOCH_ERR_ARG;
  if ((b->have & 7u) != 7u)
    return bfail(b, EPOCH_ERR_ORDER, "set models, trees and tip data before evaluating");
  if (!b->d_dh) {  // the gradient's buffers, on first use
    const size_t chain = (size_t)b->n_sm * kMaxCtasPerSm * kMaxWarps * 2 * b->Emax * b->K;
    BCK(balloc(&b->d_ex, b->total_internal), "cudaMalloc(exponents)");
    BCK(balloc(&b->d_dseg, (size_t)b->total_nodes * b->Emax), "cudaMalloc(segment terms)");
    BCK(balloc(&b->d_chain, chain), "cudaMalloc(forward vectors)");
    BCK(balloc(&b->d_dh, b->total_nodes), "cudaMalloc(height gradient)");
    BCK(balloc(&b->d_db, b->total_bnd), "cudaMalloc(boundary gradient)");
    BCK(balloc(&b->d_dbot, b->total_nodes), "cudaMalloc(bottom terms)");
    BCK(balloc(&b->d_span, b->total_nodes), "cudaMalloc(segment spans)");
  }
  if (!b->gwarps) {
    epoch_status s = forest_tune<true>(b, b->gwarps, b->gctas_per_sm);
    if (s != EPOCH_OK) return s;
  }
  epoch_status s = forest_replay<true>(b, b->ggraph, b->gwarps, b->gctas_per_sm);
  b->grad_valid = s == EPOCH_OK;
  return s;
}

epoch_status epoch_batch_read(epoch_batch *b, double *lnL) {
  if (!b || !lnL) return EPOCH_ERR_ARG;
  BCK(cudaMemcpyAsync(lnL, b->d_lnl, sizeof(double) * b->T, cudaMemcpyDeviceToHost, b->stream),
      "cudaMemcpyAsync(lnL)");
  BCK(cudaMemcpyAsync(b->h_status, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, b->stream),
      "cudaMemcpyAsync(status)");
  BCK(cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
  if (*b->h_status) {
    const int st = *b->h_status;
    BCK(cudaMemsetAsync(b->d_status, 0, sizeof(int), b->stream), "cudaMemsetAsync(status)");
    return bfail(b, EPOCH_ERR_NUMERIC, (st & FS_TERMS) ? "uniformisation term limit reached"
                                                       : "non-finite partial likelihood");
  }
  return EPOCH_OK;
}

epoch_status epoch_batch_read_gradient(epoch_batch *b, double *lnL, double *d_heights,
                                       double *d_boundaries) {
  if (!b || !lnL || !d_heights || (b->total_bnd > 0 && !d_boundaries)) return EPOCH_ERR_ARG;
  if (!b->grad_valid)
    return bfail(b, EPOCH_ERR_ORDER, "the last evaluation was not a gradient evaluation");
  BCK(cudaMemcpyAsync(d_heights, b->d_dh, sizeof(double) * b->total_nodes, cudaMemcpyDeviceToHost,
                      b->stream),
      "cudaMemcpyAsync(height gradient)");
  if (b->total_bnd > 0)
    BCK(cudaMemcpyAsync(d_boundaries, b->d_db, sizeof(double) * b->total_bnd,
                        cudaMemcpyDeviceToHost, b->stream),
        "cudaMemcpyAsync(boundary gradient)");
  return epoch_batch_read(b, lnL);
}

epoch_status epoch_batch_launch_shape(const epoch_batch *b, int *warps_per_cta, int *ctas_per_sm) {
  if (!b) return EPOCH_ERR_ARG;
  if (warps_per_cta) *warps_per_cta = b->warps;
  if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm;
  return EPOCH_OK;
}

}  // extern "C"
